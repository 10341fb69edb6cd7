/*
 * cg.h -- C ABI of libcg: parallel-rejection kinetic Monte Carlo of the 2D
 * lattice Coulomb glass on one NVIDIA GB300 (sm_103a).
 *
 * Method: E.E. Ferrero, A.B. Kolton, M. Palassini, "Parallel kinetic Monte
 * Carlo simulation of Coulomb glasses".  The model is the Hamiltonian of
 * Eq. 1 on an L x L torus with minimum-image distances (section "Results for
 * the lattice model in two dimensions"); the dynamics is the mixed PR
 * algorithm (section "Hopping conduction in the Coulomb glass", steps 1-3):
 * M labels per round propose hops i -> j drawn from the tunnelling factor of
 * Eq. 2 by tower sampling, each is tested with the activation factor
 * min[1, exp(-dH/T)], the lowest accepting label is executed, and the N
 * local energies eps are updated (step 3b).
 *
 * Conventions shared by every entry point
 *   - Sites are numbered s = y*L + x, x, y in [0, L).
 *   - All pointers named *_host point to host memory owned by the caller;
 *     the library copies from/to them and keeps no reference.
 *   - Device memory is owned by the library (cudaMalloc) unless the handle
 *     was created over a caller workspace (cg_create_batch_ws), in which case
 *     the caller owns that workspace and must keep it alive until
 *     cg_destroy returns.
 *   - Every int-returning call returns CG_OK (0) or a negative CG_E* code and
 *     never throws; cg_last_error() gives a message for the calling thread's
 *     last failure.  A handle whose call returned CG_ECUDA should be
 *     destroyed.
 *   - Calls on one handle must not overlap (one host thread at a time).
 */
#ifndef CG_H
#define CG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CG_OK 0
#define CG_EINVAL (-1)   /* a parameter is out of range; nothing changed      */
#define CG_ENOMEM (-2)   /* device or host allocation failed                  */
#define CG_ECUDA (-3)    /* a CUDA call failed; the message names it          */
#define CG_ETIMEOUT (-4) /* a bounded device wait ran out                     */
#define CG_ESTUCK (-5)   /* max rounds per hop reached without an accept; the
                            state is valid and the failed rounds are counted */
#define CG_ESTATE (-6)   /* a state passed in is inconsistent                 */

#define CG_FP64 0        /* eps in binary64: bit-exact with the serial chain  */
#define CG_FP32 1        /* eps in binary32 with a periodic binary64 refresh  */

/* cg_opts.time_mode */
#define CG_TIME_DETERMINISTIC 0
#define CG_TIME_GAUSSIAN 1

#define CG_REFRESH_AUTO 0
#define CG_REFRESH_FP64 1  /* direct G (n - nu) in binary64                   */
#define CG_REFRESH_BF16X2 2 /* split-BF16 hi+lo tensor-core contraction over
                               the replicas of one L                          */
#define CG_REFRESH_FFT 3   /* the convolution theorem: binary32 FFTs of
                               n - nu, two replicas per complex transform,
                               times DFT(1/r); L = 2^m or 3 2^m            */

typedef struct cg_handle cg_handle;

/* One disorder replica: the parameters of Eq. 1 and Eq. 2.
 *   L      lattice side, even, 4 <= L; N = L*L sites
 *   nu     filling factor, 0 < nu < 1, nu*N an integer (electrons)
 *   W      full width of the site-energy interval: phi ~ U[-W/2, W/2]
 *   xi     localisation length (> 0) in the tunnelling factor exp(-2r/xi)
 *   r_max  hop cut-off radius, 1 <= r_max < L/2 (hops inside the disk)
 *   T      temperature (> 0)
 *   E      field along x; dH of a hop contains -E*dx
 *   seed   Philox key (64 bits)
 *   replica  Philox counter word 3 of every draw of this replica
 *   dim    0 or 2: the L x L square lattice of the paper; 3: the L x L x L
 *          cubic lattice (the three-dimensional extension named in the
 *          paper's conclusions; L <= 64, hop ball dx^2+dy^2+dz^2 <= r_max^2,
 *          one CTA per replica or, when eps does not fit one, a cluster
 *          of 2, 4 or 8 CTAs splitting it by z-planes; binary32 refreshed
 *          on the tensor cores when L^3 is a multiple of 128, else in
 *          binary64)
 *   sites  CG_SITES_LATTICE (0), or CG_SITES_RANDOM: the random-site
 *          Coulomb glass, N = L^2 sites at Philox positions in the L x L
 *          periodic box (counter (s, 3, 0xFFFFFFFF, replica): x = L (x0 +
 *          1/2) 2^-32, y = L (x1 + 1/2) 2^-32), minimum-image 1/r, hop
 *          partners j != i with r_ij <= r_max drawn by an integer tower of
 *          weights floor(2^32 exp(-2 r / xi) / Zmax) (Zmax the largest
 *          per-site sum), Gamma = N Zmax, the real minimum-image dx in the
 *          field term and no dipole counter (P stays 0).  Binary64, single
 *          hops, deterministic time (else CG_EINVAL); N <= 131072 (L <= 362;
 *          partner lists below 2^16 pairs); one CTA per replica, or, when
 *          eps (8 N bytes) does not fit one or cluster_size forces it, a
 *          cluster of 2, 4 or 8 CTAs, CTA r owning the eps of sites
 *          [r Nc, (r+1) Nc), Nc = ceil(N / C) rounded up to a multiple of
 *          32 (any even L).  The N x N coupling matrix (8 N^2 bytes) lives
 *          in device memory (CG_ENOMEM when it does not fit).           */
typedef struct {
    int32_t L;
    int32_t r_max;
    double nu, W, xi, T, E;
    uint64_t seed;
    uint32_t replica;
    int32_t dim;
    int32_t sites;
    int32_t reserved_;   /* 0 */
} cg_replica_desc;

#define CG_SITES_LATTICE 0
#define CG_SITES_RANDOM 1

/* Options of a handle.  Zero-initialised means: FP64, no refresh, automatic
 * launch shape, 2^32 rounds per hop before CG_ESTUCK, a 10 s limit per hop,
 * device 0, a stream created by the library. */
typedef struct {
    int32_t precision;          /* CG_FP64 or CG_FP32                           */
    int32_t refresh_kind;       /* CG_REFRESH_*                                 */
    uint32_t refresh_every;     /* FP32: hops between refreshes, 0 = never      */
    int32_t block_threads;      /* 0 = automatic; else 256, 384, 512 or 1024  */
    uint64_t max_rounds_per_hop;/* 0 = 2^32                                     */
    int32_t device;             /* CUDA device ordinal                          */
    int32_t use_graph;          /* 1: cg_run replays a captured CUDA graph      */
    void *stream;               /* cudaStream_t to launch on; NULL = own stream */
    uint32_t hop_timeout_ms;    /* wall-clock limit of one hop on the device
                                   (0 = 10000 ms); past it the launch stops
                                   with CG_ETIMEOUT, the state stays valid    */
    int32_t cluster_size;       /* CTAs per replica: 0 = automatic (one CTA when
                                   the replica fits its shared memory, else the
                                   smallest of 2, 4, 8 that fits); 2, 4 or 8
                                   force a thread-block cluster that splits
                                   eps by rows (CTA r of C holds the rows
                                   [r L/2C, (r+1) L/2C) and the same rows
                                   + L/2, so L must be a multiple of 2C) or
                                   by z-planes on the cubic lattice (L a
                                   multiple of C), or by site index on random
                                   sites (any even L)                          */
    int32_t time_mode;          /* CG_TIME_DETERMINISTIC (0): t = attempts/Gamma;
                                   CG_TIME_GAUSSIAN: each executed hop adds a
                                   Gaussian dt of mean m/Gamma and standard
                                   deviation sqrt(m)/Gamma, m = (p-1)M + q
                                   (mixed PR algorithm, step 3c), clamped at 0 */
    int32_t pair_rmax;          /* two-electron hops (pair_frac > 0): the second
                                   electron sits at an offset e with
                                   0 < |e| <= pair_rmax from the first, and the
                                   reverse move's offset must obey the same
                                   bound; 1 <= pair_rmax, 2 pair_rmax < L      */
    double pair_frac;           /* fraction p2 in [0, 1) of the labels that
                                   propose a two-electron hop (the paper's
                                   multi-electron hops, named in its
                                   conclusions as an extension): a label is a
                                   pair proposal iff its fourth Philox word is
                                   below floor(p2 2^32).  0 = single hops only.
                                   Square and cubic lattices, one CTA or a
                                   cluster, both clocks; Gamma becomes
                                   N Z / (1 - floor(p2 2^32) 2^-32)            */
} cg_opts;

/* Counters of one replica (step 3 of the mixed PR algorithm). */
typedef struct {
    uint64_t rounds;     /* global round counter r (every round, accepted or not) */
    uint64_t hops;       /* executed hops                                         */
    uint64_t attempts;   /* serial-equivalent attempts: (p-1) M + q per hop       */
    uint64_t evaluated;  /* labels actually evaluated on the GPU                  */
    int64_t P;           /* dipole moment sum_i n_i x_i, unwrapped by hop dx      */
    double energy;       /* H of Eq. 1 (field term with the unwrapped P)          */
    double time;         /* CG_TIME_GAUSSIAN: the accumulated stochastic time;
                            CG_TIME_DETERMINISTIC: 0 (time is attempts/Gamma)     */
} cg_counters;

/* Observables of one replica. */
typedef struct {
    cg_counters c;
    double time;              /* attempts / Gamma, or the stochastic time of
                                 CG_TIME_GAUSSIAN                             */
    double Gamma;             /* N * sum_d exp(-2|d|/xi) over the hop disk     */
    double acceptance;        /* hops / attempts                              */
    double energy_per_site;   /* energy / N                                   */
    double max_eps_err_last_refresh; /* FP32: max |eps - eps_refreshed| seen
                                        just before the last refresh          */
    uint64_t refreshes;       /* refreshes done                                */
    uint64_t cycles_reject;   /* SM clock cycles spent proposing/testing       */
    uint64_t cycles_update;   /* SM clock cycles spent in the eps update       */
} cg_obs;

/* One point of the log-spaced trace (cg_set_trace). */
typedef struct {
    uint64_t attempts;   /* serial-equivalent attempts when recorded                       */
    uint64_t hops;
    int64_t P;           /* dipole moment (unwrapped)                                      */
    double energy;
    double time;         /* attempts/Gamma, or the stochastic time of CG_TIME_GAUSSIAN     */
} cg_trace_point;

/* One executed hop (diagnostics; see cg_run_logged). */
typedef struct {
    uint32_t i, j;       /* origin, destination                        */
    uint32_t q;          /* 1-based label of the hop in its round      */
    uint32_t p;          /* rounds used for this hop                   */
    uint64_t round;      /* round counter of the accepting round       */
    int32_t dx, dy;      /* hop vector                                 */
    double dE;           /* dH of the hop (binary64; of both electrons
                            for a two-electron hop)                    */
    uint32_t k, l;       /* second electron of a two-electron hop:
                            origin, destination; 0xFFFFFFFF otherwise  */
    int32_t dx2, dy2;    /* its hop vector; 0 otherwise                */
} cg_hop;

/* ---------------------------------------------------------------------- */

/* Create one FP64 replica with replica index 0 (the arguments of
 * cg_replica_desc).  Builds the tables, draws disorder phi and the initial
 * random occupation from Philox(seed), computes eps from scratch.
 * Returns NULL on error (cg_last_error). */
cg_handle *cg_create(int L, double nu, double W, double xi, int r_max,
                     double T, double E, uint64_t seed);

/* Create R replicas (any mix of L) sharing one stream and one option set.
 * reps: R host descriptors; opts may be NULL (defaults). */
cg_handle *cg_create_batch(int R, const cg_replica_desc *reps,
                           const cg_opts *opts);

/* Bytes of device workspace cg_create_batch_ws needs for these replicas. */
size_t cg_workspace_bytes(int R, const cg_replica_desc *reps,
                          const cg_opts *opts);

/* As cg_create_batch, but every device buffer is carved from the caller's
 * workspace (device pointer, 256-byte aligned, ws_bytes >= cg_workspace_bytes);
 * the library then calls no cudaMalloc for this handle. */
cg_handle *cg_create_batch_ws(int R, const cg_replica_desc *reps,
                              const cg_opts *opts, void *workspace,
                              size_t ws_bytes);

void cg_destroy(cg_handle *h);

/* Message of the calling thread's last error ("" if none). */
const char *cg_last_error(void);

int cg_num_replicas(const cg_handle *h);
int cg_num_sites(const cg_handle *h, int replica);

/* Positions of a random-site replica's N sites (CG_SITES_RANDOM; the
 * Philox positions of the descriptor's definition, in the L x L box): x into
 * x_host[0..N), y into y_host[0..N) (caller-owned host arrays).  With the
 * occupation from cg_read_state they give the real dipole sum n_s x_s, which
 * the counters do not keep on random sites.  CG_EINVAL for a null handle or
 * output, a replica out of range or a lattice replica; no device work. */
int cg_site_positions(const cg_handle *h, int replica, double *x_host, double *y_host);

/* Advance every replica by n_hops executed hops with M labels per round
 * (mixed PR algorithm, steps 1-3; 1 <= M <= 2^24, or M = 0 for each lattice
 * size's own M: 4096 unless cg_autotune chose another).  Blocks until the
 * work is done.  FP32 handles refresh eps every refresh_every hops.  Replicas
 * of different L run as concurrent launches (one stream each, forked from and
 * joined to the handle's stream); with opts.use_graph the launches of each
 * distinct (n_hops, M, refresh phase) are captured once in a CUDA graph and
 * replayed.  Returns CG_ESTUCK if some replica reached max_rounds_per_hop;
 * other replicas still completed their hops. */
int cg_run(cg_handle *h, uint64_t n_hops, uint32_t M);

/* cg_run without the final wait: the work is queued on the handle's stream
 * and cg_sync() waits for it and returns its status. */
int cg_run_async(cg_handle *h, uint64_t n_hops, uint32_t M);
int cg_sync(cg_handle *h);

/* cg_run that also records every executed hop: log_host receives
 * R * n_hops entries, replica-major. */
int cg_run_logged(cg_handle *h, uint64_t n_hops, uint32_t M, cg_hop *log_host);

/* Copy one replica's state to host buffers (NULL pointers are skipped): the
 * configuration and local energies of the mixed PR algorithm (section
 * "Hopping conduction in the Coulomb glass": occupations n_i, the site
 * energies phi_i of Eq. 1 and eps_i = phi_i + sum_j (n_j - nu)/r_ij below
 * Eq. 2) and the counters of step 3.
 *   n_host    N bytes (0/1)
 *   eps_host  N doubles (FP32 eps widened exactly)
 *   phi_host  N doubles
 *   c_host    the counters (rounds, hops, attempts (p-1)M + q summed over
 *             hops, P of Eq. 3, the running energy of Eq. 1)
 * Waits for the handle's queued work first.  CG_EINVAL for a null handle or
 * a replica out of range, CG_ECUDA on a CUDA error. */
int cg_read_state(cg_handle *h, int replica, uint8_t *n_host, double *eps_host,
                  double *phi_host, cg_counters *c_host);

/* Overwrite one replica's state.  n_host (N bytes 0/1, nu*N ones) is
 * required; phi_host replaces the disorder when non-NULL; eps_host sets eps
 * when non-NULL, otherwise eps is rebuilt from scratch; c_host sets the
 * counters when non-NULL, otherwise the counters restart at 0 with the energy
 * and dipole recomputed.  Returns CG_ESTATE for a bad occupation. */
int cg_write_state(cg_handle *h, int replica, const uint8_t *n_host,
                   const double *eps_host, const double *phi_host,
                   const cg_counters *c_host);

/* Observables of one replica (cg_obs): its counters, the time t = attempts /
 * Gamma of the deterministic clock (the rule behind the paper's Fig. 3) or
 * the stochastic clock of step 3c, Gamma = N sum_d exp(-2|d|/xi) of the mixed
 * algorithm, the acceptance hops / attempts (the A of the section "Parallel
 * rejection algorithm"), the energy per site of Eq. 1, the last refresh's
 * eps error and the kernels' phase clocks.  Waits for the handle's queued
 * work first.  CG_EINVAL for a null handle or output or a replica out of
 * range, CG_ECUDA on a CUDA error. */
int cg_observables(cg_handle *h, int replica, cg_obs *out);

/* Rebuild eps of every replica from scratch now, from its definition below
 * Eq. 2: eps_s = phi_s + sum_{t != s} (n_t - nu) / r_st.  CG_FP64 handles
 * recompute it in the serial summation order (bit-identical to a fresh
 * start).  CG_FP32 handles record the largest |eps_fp32 - eps_new|
 * (cg_obs.max_eps_err_last_refresh) and store eps_new rounded to binary32,
 * where eps_new comes from one of three paths:
 *   - a group of replicas of one L = 2^m (4 <= L <= 1024) or 3 2^m (6 <= L
 *     <= 192) (CG_REFRESH_AUTO or CG_REFRESH_FFT): the convolution theorem,
 *     eps - phi = IDFT(DFT(n - nu) DFT(1/r)) on the periodic lattice,
 *     radix-2 (and one radix-3) transforms in binary32 with two replicas per
 *     complex transform (DFT(1/r) is real), DFT(1/r) and the
 *     twiddles from binary64 on the host, phi added in binary64 (error below
 *     2e-5 up to L = 256 square and L = 64 cubic, measured against the
 *     definition);
 *   - otherwise, a group of replicas of one L whose N is a multiple of 128
 *     (CG_REFRESH_AUTO with at least 8 replicas, or CG_REFRESH_BF16X2): the
 *     tensor-core contraction, the
 *     1/r table split into two BF16 terms (binary16 terms of 2^10/r on the
 *     cubic lattice), the +-1 occupations exact in that format, products
 *     accumulated in binary32 by the tensor cores over K ranges of at most
 *     2048 sites and the partial sums and phi added in binary64 (error below
 *     5e-5 at L <= 128, measured against the definition);
 *   - otherwise (or CG_REFRESH_FP64): a direct sum in binary64.
 * Blocks until done. */
int cg_refresh(cg_handle *h);

/* cg_refresh queued on the handle's stream without waiting (cg_sync waits). */
int cg_refresh_async(cg_handle *h);

/* The tensor-core refresh of cg_refresh for callers that cannot allocate
 * device memory (a host program that owns the allocator, a service whose
 * device footprint is fixed after start-up, code that must make no
 * allocation call).  The paper has no counterpart: this is a deployment
 * variant of the refresh, not a step of the method.
 *
 * Rebuilds eps of R binary32 replicas of one side L from their occupations:
 * eps_s = phi_s + sum_{t != s} (n_t - nu) / r_st, computed exactly as
 * cg_refresh computes it for a tensor-core batch (split-BF16 contraction,
 * binary64 reduction), and reports max |eps_old - eps_new| per replica.
 *   L        even, 16 <= L <= 1024, L*L a multiple of 128
 *   R        1 <= R <= 512
 *   nu       filling factor of every replica
 *   occ      device, R x ceil(L*L/32) words, replica-major; bit s%32 of word
 *            s/32 is the occupation of site s
 *   phi      device, R x L*L binary64 site energies
 *   eps      device, R x L*L binary32; read (old eps) and overwritten
 *   max_err  device, R binary64 outputs, or NULL
 *   stream   cudaStream_t to run on (NULL: the legacy default stream)
 * All pointers are owned by the caller.  The call allocates nothing: its
 * scratch is one static device array of 32 MiB that every GPU loading the
 * library holds until the process exits.  A call needs (2 + 4 k) N R_pad
 * bytes of it for the contraction (R_pad = R rounded up to a multiple of 16,
 * k the K split: 8 at L = 32, 64, 96 and 128, 10 at L = 160, 11 at L = 176)
 * plus 352 bytes per replica and the split 1/r table, each part rounded up
 * to 256 bytes.  The largest accepted R is 512 up to L = 48, 240 at L = 64,
 * 224 at L = 80, 96 at L = 96, 80 at L = 112, 48 at L = 128, 32 at L = 144
 * and 16 at L = 160 and 176; every L from 192 up needs more than 32 MiB even
 * for R = 1.  Larger requests return CG_EINVAL with the limit in the
 * message.  The first call on a device (and again after the device's context
 * changed, e.g. after cudaDeviceReset) looks up the array's device address
 * and should come before any stream capture.  Every call shares the array and
 * leaves its contents behind: calls that overlap on the GPU (other streams,
 * other host threads, same device) race and must be serialised by the
 * caller.  The call waits for its stream before returning.
 * Returns CG_OK, CG_EINVAL, CG_ECUDA, or CG_ETIMEOUT if a bounded device wait
 * ran out. */
int cg_refresh_tc_noalloc(int L, int R, double nu, const unsigned int *occ,
                          const double *phi, float *eps, double *max_err,
                          void *stream);

/* Peak-rate microbenchmarks of the device (no handle needed):
 *   kind 0: shared-memory read-modify-write bandwidth of 32-bit words, bytes/s
 *   kind 1: binary64 add throughput, adds/s
 *   kind 2: shared-memory read-modify-write bandwidth of 64-bit words, bytes/s
 *   kind 3: Philox-4x32-10 blocks/s of the PR kernels' label generator (the
 *           ceiling of the rejection phase: one block per evaluated label;
 *           section "Parallel rejection algorithm", 3M random numbers per
 *           round on the GPU)
 * summed over all SMs;
 *   kind 4, 5, 6: seconds per cluster barrier of 2, 4 or 8 CTAs of 1024
 *           threads (one CTA per SM, all SMs busy), the fixed cost of the
 *           cluster kernels' chunks and hops;
 *   kind 7: seconds per CTA barrier of 1024 threads (one CTA per SM);
 * result written to *result.  CG_EINVAL for another kind, CG_ECUDA on a
 * CUDA error. */
int cg_microbench(int kind, int device, double *result);

/* Log-spaced trace of the dipole moment P and the energy, from which the
 * conductivity sigma(t) = (1 / N E) dP/dt of Eq. 3 is estimated (P(t) and
 * its relaxation are the paper's Fig. 3 observables).  After this call every
 * replica records a point at the first executed hop whose time reaches
 * t_k = first_time * 10^(k / points_per_decade) (time in units of tau_0,
 * t = attempts / Gamma), up to `capacity` points; the first point is the
 * state at the call.  Allocates per-replica device buffers (cudaMalloc, also
 * for workspace handles); a later call restarts the trace. */
int cg_set_trace(cg_handle *h, double first_time, double points_per_decade, int capacity);

/* Copy up to `cap` recorded points of one replica into out_host; returns
 * the number of points copied (>= 0) or a negative CG_E* code. */
int cg_read_trace(cg_handle *h, int replica, cg_trace_point *out_host, int cap);

/* Launch-shape autotuner.  The parallel-rejection section recommends M near
 * 1/A but larger than the number of concurrent threads; the best M and launch
 * shape depend on the GPU, so for every group of replicas with one L this
 * times the persistent launch for every cluster size (CTAs per replica: 1
 * when eps fits one CTA, and each of 2, 4, 8 that fits, on lattices only
 * those whose row or plane split divides L; only the forced size when
 * cg_opts.cluster_size was set), CTA sizes 256, 384, 512, 1024 (those the
 * kernel takes) and M in
 * {1024, 4096, 16384, 65536}, over hops_per_trial hops (0: 256) on a copy of the
 * group's state.  A trial counts only when every replica of the group
 * completed its hops.  The state is restored bit for bit after each trial
 * and the fastest shape is kept (cg_run with M = 0 then uses its M).  With
 * $CG_TUNE_CACHE naming a JSON file, cached shapes are reused and new ones
 * added.  Allocates a temporary device snapshot; captured graphs are
 * dropped. */
int cg_autotune(cg_handle *h, uint32_t hops_per_trial);

/* Groups of replicas sharing one L (one persistent launch each). */
int cg_num_groups(const cg_handle *h);
int cg_group_shape(const cg_handle *h, int index, int *L, int *threads,
                   unsigned int *M, int *cluster);

/* Replica indices of group `group` (the replicas with its L and
 * dimension, ascending) written to replicas_out, which must hold
 * cg_num_replicas entries; returns their count (>= 1), or CG_EINVAL for a
 * bad group or a NULL output.  The paper has no counterpart: this and the
 * next two calls are the batch form of the state I/O (checkpoint/resume of
 * a whole batch). */
int cg_group_replicas(const cg_handle *h, int group, int *replicas_out);

/* Read the state of every replica of one group in one copy per array
 * (device order = cg_group_replicas order; NULL pointers are skipped):
 *   occ_words_host  count * ceil(N/32) words, bit s of word s/32 = n_s;
 *   eps_host        count * N values in the handle's precision (double for
 *                   CG_FP64, float for CG_FP32), not widened;
 *   c_host          count counter records.
 * Pinned host buffers make the copies asynchronous DMA; the call blocks
 * until they are done.  CG_EINVAL for a bad group, CG_ECUDA on a CUDA error. */
int cg_read_group_state(cg_handle *h, int group, uint32_t *occ_words_host,
                        void *eps_host, cg_counters *c_host);

/* Write the same arrays back (NULL pointers are skipped).  Occupations and
 * eps are stored as given: eps is not recomputed (cg_refresh rebuilds it
 * from the occupation); every replica must keep nu*N electrons and no bit
 * beyond site N-1, else CG_ESTATE and nothing is written.  The counter
 * records replace the public counters; the library's own per-replica fields
 * (chunk statistics, refresh record, trace state, phase clocks) are kept.
 * Blocks until the copies are done. */
int cg_write_group_state(cg_handle *h, int group, const uint32_t *occ_words_host,
                         const void *eps_host, const cg_counters *c_host);

/* Test-only constant-acceptance mode: every label accepts iff u < A0, the
 * configuration is never changed, the counters advance.  A0 < 0 turns the
 * mode off.  CG_EINVAL on a handle with random-site replicas. */
int cg_set_toy_acceptance(cg_handle *h, double A0);

/* Exported device helpers for tests: evaluate Philox-4x32-10 and the
 * acceptance exponential on the GPU for n inputs (host arrays in/out). */
int cg_debug_philox(const uint32_t *ctr_host, const uint32_t *key_host,
                    uint32_t *out_host, int n);
int cg_debug_exp(const double *x_host, double *out_host, int n);

/* Test-only: the standard normal deviate of executed hop hops_host[k] of
 * replica replica_host[k] under seed seed_host[k] (Box-Muller on the Philox
 * block of counter (hop lo, hop hi, 0xFFFFFFFE, replica), as the kernels draw
 * it for CG_TIME_GAUSSIAN), on the GPU for n inputs (host arrays). */
int cg_debug_gauss(const uint64_t *seed_host, const uint32_t *replica_host,
                   const uint64_t *hops_host, double *z_host, int n);

/* Test-only: the PR kernels' tower sampler (guide table + thresholds of
 * replica `replica`, section "Hopping conduction in the Coulomb glass": hop
 * vector by tower sampling) on the GPU for n 32-bit words x1 (host arrays).
 * v_host[k] = the smallest vector index v with x1 < C_v, C the integer
 * cumulative weights in the table's order, or -1 for a null proposal
 * (x1 >= C_{V-1}).  Returns CG_EINVAL for bad arguments or a random-site
 * replica (it draws from its partner lists), CG_ECUDA on a CUDA error;
 * allocates and frees device memory internally. */
int cg_debug_tower(cg_handle *h, int replica, const uint32_t *x1_host, int32_t *v_host, int n);

/* Density of states of the local energies: the histogram g(eps) whose
 * Coulomb gap the paper discusses (section "Results for the lattice model in
 * two dimensions", single-particle density of states).  For the sites s of
 * replicas first .. first+count-1 (handle order), with x = (eps_s - lo) *
 * (nbins / (hi - lo)) (eps widened to binary64, each operation rounded once,
 * the scale computed once in binary64): a site with eps_s >= lo and
 * x < nbins adds 1 to counts_dev[floor(x)]; other sites are not counted.
 *   counts_dev  DEVICE array of nbins uint64, owned by the caller; the
 *               counts are ADDED to it (zero it first; repeated calls sum
 *               snapshots over time without leaving the device)
 *   nbins       1 .. 4096;  lo < hi, both finite
 * Enqueued on the handle's stream after its pending work; returns without
 * waiting (read counts_dev after cg_sync).  Allocates nothing.  CG_EINVAL
 * for bad arguments, CG_ECUDA on a launch error. */
int cg_eps_histogram(cg_handle *h, int first, int count, int nbins, double lo, double hi,
                     uint64_t *counts_dev);

/* Library version string. */
const char *cg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CG_H */
