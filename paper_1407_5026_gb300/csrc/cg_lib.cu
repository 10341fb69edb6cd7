// cg_lib.cu -- host side of libcg: parameter checks, tables, disorder and
// initial state, device memory, launch orchestration and the C ABI of
// include/cg.h.
//
// Set-up follows the model of Eq. 1 on an L x L torus with minimum-image
// distances (section "Results for the lattice model in two dimensions"):
//   * folded 1/r table over |dx|, |dy| in [0, L/2], zero at the origin;
//   * hop vectors: all (dx, dy) with 0 < dx^2 + dy^2 <= r_max^2, dy outer,
//     dx inner, both ascending; tunnelling weights w = exp(-2r/xi) (Eq. 2),
//     Z = sum w, integer tower weights floor(2^32 w / Z) and their running
//     sums (tower sampling of the mixed algorithm);
//   * Gamma = N Z, the total tunnelling rate; time = attempts / Gamma;
//   * phi_s = W (u - 1/2) with u = (x0 + 1/2) 2^-32 from Philox counter
//     (s, 1, 0xFFFFFFFF, replica): site energies uniform on a width-W interval;
//   * initial random configuration: sites sorted by (x0 of counter
//     (s, 2, 0xFFFFFFFF, replica), s), the first nu N occupied.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "cg_device.cuh"
#include "cg_internal.h"

using namespace cg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CG_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(CG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

// exp(x), -745 < x <= 0: Cody-Waite reduction with ln 2 = LN2_HI + LN2_LO and
// the degree-13 Taylor polynomial, exactly as the device's acceptance
// exponential but without its cut-off (used for the tunnelling weights).
double host_exp(double x)
{
    const double kd = std::nearbyint(x * 0x1.71547652b82fep+0);
    const double r = (x - kd * 0x1.62e42ffp-1) - kd * -0x1.718432a1b0e26p-35;
    static const double inv_fact[14] = {
        1.0, 1.0, 0x1.0p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
        0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
        0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
        0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    double p = inv_fact[13];
    for (int n = 12; n >= 0; --n) {
        const double t = p * r;
        p = t + inv_fact[n];
    }
    return std::ldexp(p, (int)kd);
}

// Round-to-nearest-even binary32 -> BF16 (finite inputs), and back.
uint32_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    return (u + 0x7fffu + lsb) >> 16;
}

float bf16_to_float(uint32_t h)
{
    const uint32_t u = h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Round-to-nearest-even of a finite double with |v| < 65520 to IEEE binary16
// bits (subnormals included), and back.
uint32_t f16_rne(double v)
{
    const uint32_t sign = v < 0 ? 0x8000u : 0u;
    const double a = std::fabs(v);
    if (a == 0.0) return sign;
    int e;
    std::frexp(a, &e);                         // a = m 2^e, m in [1/2, 1)
    int E = e - 1 < -14 ? -14 : e - 1;         // binade; below 2^-14 the subnormal spacing
    double k = std::nearbyint(std::ldexp(a, 10 - E));   // units of 2^(E-10), ties to even
    if (k >= 2048.0) { k = 1024.0; E += 1; }   // rounded up into the next binade
    const uint32_t bits = k < 1024.0 ? (uint32_t)k
                                     : ((uint32_t)(E + 15) << 10) | ((uint32_t)k - 1024u);
    return sign | bits;
}

double f16_to_double(uint32_t h)
{
    const int ex = (int)((h >> 10) & 31u), man = (int)(h & 1023u);
    const double v = ex == 0 ? std::ldexp((double)man, -24) : std::ldexp((double)(man + 1024), ex - 25);
    return (h & 0x8000u) ? -v : v;
}

struct Tables {
    int L = 0, r_max = 0, H1 = 0, V = 0;
    double xi = 0, Z = 0, C0 = 0;
    int dim = 2;                      // 2: square lattice, 3: cubic lattice
    std::vector<double> t64;
    std::vector<float> t32;
    std::vector<unsigned> thr;
    std::vector<int> disp;
    std::vector<double> tinvd;
    std::vector<unsigned short> guide;
    std::vector<uint32_t> split;      // hi | lo << 16 of each 1/r entry: BF16 of 1/r on the
                                      // square lattice, binary16 of 2^10 / r on the cubic one
    // cubic lattice: the folded table's values indexed by r^2 = fx^2 + fy^2 +
    // fz^2 (3 (L/2)^2 + 1 entries; 0 where r^2 is no sum of three squares)
    std::vector<double> r2_64;
    std::vector<float> r2_32;
    double *d_r2_64 = nullptr;
    float *d_r2_32 = nullptr;
    // the FFT refresh (binary32 handles, power-of-two L): DFT(g) / N of the
    // minimum-image 1/r (real: g is even) and the twiddles exp(-2 pi i k/L)
    std::vector<float> ghat;
    std::vector<float2> tw;
    float *d_ghat = nullptr;
    float2 *d_tw = nullptr;
    unsigned short *d_guide = nullptr;
    uint32_t *d_split = nullptr;
    double *d_t64 = nullptr;
    float *d_t32 = nullptr;
    unsigned *d_thr = nullptr;
    int *d_disp = nullptr;
    double *d_tinvd = nullptr;
};

int build_tables(Tables &t, int L, double xi, int r_max, int dim)
{
    t.L = L; t.xi = xi; t.r_max = r_max; t.H1 = L / 2 + 1; t.dim = dim;
    const int H1 = t.H1, Hz = dim == 3 ? H1 : 1;
    // folded 1/r table, [(fz H1 + fy) H1 + fx], 0 at the origin
    t.t64.assign((size_t)Hz * H1 * H1, 0.0);
    for (int fz = 0; fz < Hz; ++fz)
        for (int fy = 0; fy < H1; ++fy)
            for (int fx = 0; fx < H1; ++fx)
                t.t64[((size_t)fz * H1 + fy) * H1 + fx] =
                    (fx == 0 && fy == 0 && fz == 0)
                        ? 0.0 : 1.0 / std::sqrt((double)(fx * fx + fy * fy + fz * fz));
    t.t32.resize(t.t64.size());
    for (size_t k = 0; k < t.t64.size(); ++k) t.t32[k] = (float)t.t64[k];
    if (dim == 3) {
        // 1/r depends on r^2 alone, so each r^2 takes the folded entry's
        // bits (every offset with that r^2 holds the same value)
        const int h = L / 2;
        t.r2_64.assign((size_t)3 * h * h + 1, 0.0);
        t.r2_32.assign(t.r2_64.size(), 0.0f);
        for (int fz = 0; fz < H1; ++fz)
            for (int fy = 0; fy < H1; ++fy)
                for (int fx = 0; fx < H1; ++fx) {
                    const size_t k = ((size_t)fz * H1 + fy) * H1 + fx;
                    const int q = fx * fx + fy * fy + fz * fz;
                    t.r2_64[q] = t.t64[k];
                    t.r2_32[q] = t.t32[k];
                }
    }
    // two-term split of 1/r for the tensor-core refresh.  Square lattice:
    // hi = bf16(T), lo = bf16(T - hi), so T - hi - lo is below 2^-16 of T.
    // Cubic lattice, where sum_t G_st^2 is about eight times larger and that
    // residual would reach 1e-4 on eps at L = 32: binary16 terms of
    // T' = 2^10 T (hi = f16(T'), lo = f16(T' - hi), residual below 2^-21 of
    // T'; the scale keeps lo out of the subnormal range), undone in binary64
    // after the contraction.
    t.split.resize(t.t64.size());
    for (size_t k = 0; k < t.t64.size(); ++k) {
        if (dim == 3) {
            const double Ts = std::ldexp(t.t64[k], kTcF16Log2Scale);
            const uint32_t hi = f16_rne(Ts);
            const uint32_t lo = f16_rne(Ts - f16_to_double(hi));
            t.split[k] = hi | (lo << 16);
        } else {
            const uint32_t hi = bf16_rne((float)t.t64[k]);
            const double rest = t.t64[k] - (double)bf16_to_float(hi);
            const uint32_t lo = bf16_rne((float)rest);
            t.split[k] = hi | (lo << 16);
        }
    }
    // sum_{t != s} 1/r_st is the same for every s: every displacement once
    double C0 = 0.0;
    const int Lz = dim == 3 ? L : 1;
    for (int dz = 0; dz < Lz; ++dz)
        for (int dy = 0; dy < L; ++dy)
            for (int dx = 0; dx < L; ++dx)
                C0 += t.t64[((size_t)fold_axis(dz, Lz) * H1 + fold_axis(dy, L)) * H1 +
                            fold_axis(dx, L)];
    t.C0 = C0;
    // hop vectors, dz outermost (the square lattice: dz = 0 only), packed as
    // dx | dy << 16 on the square lattice and as 10-bit fields
    // dx | dy << 10 | dz << 20 on the cubic lattice
    std::vector<double> w;
    const int Rz = dim == 3 ? r_max : 0;
    for (int dz = -Rz; dz <= Rz; ++dz)
        for (int dy = -r_max; dy <= r_max; ++dy)
            for (int dx = -r_max; dx <= r_max; ++dx) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0 || r2 > r_max * r_max) continue;
                t.disp.push_back(dim == 3 ? (int)((unsigned)(dx & 0x3ff) | ((unsigned)(dy & 0x3ff) << 10) |
                                                  ((unsigned)dz << 20))
                                          : (dx & 0xffff) | (dy * 65536));
                w.push_back(host_exp(-2.0 * std::sqrt((double)r2) / xi));
                t.tinvd.push_back(
                    t.t64[((size_t)std::abs(dz) * H1 + std::abs(dy)) * H1 + std::abs(dx)]);
            }
    t.V = (int)w.size();
    double Z = 0.0;
    for (double v : w) Z = Z + v;
    t.Z = Z;
    unsigned long long run = 0;
    for (int k = 0; k < t.V; ++k) {
        const double f = (w[k] / Z) * 4294967296.0;
        const unsigned long long Wk = (unsigned long long)std::floor(f);
        if (Wk == 0)
            return fail(CG_EINVAL, "a hop vector's tower weight is below 2^-32 "
                                   "(r_max too large for xi)");
        run += Wk;
        t.thr.push_back((unsigned)(run - 1));
    }
    // guide table: smallest vector whose threshold reaches each bucket (14
    // bits); bit 15 set when a threshold lies inside the bucket (one compare
    // decides between it and the next vector), bit 14 when two or more do
    // (the sampler then keeps scanning)
    if (t.V > 0x3fff) return fail(CG_EINVAL, "more than 16383 hop vectors (r_max too large)");
    t.guide.assign(kGuide, 0);
    const int shift = 32 - kGuideBits;
    int v = 0;
    for (int b = 0; b < kGuide; ++b) {
        const unsigned long long lo = (unsigned long long)b << shift;
        const unsigned long long hi = lo + (1ull << shift) - 1;
        while (v < t.V - 1 && t.thr[v] < lo) ++v;
        const bool scan = t.thr[v] >= lo && t.thr[v] < hi;
        const bool multi = scan && v + 1 < t.V && t.thr[v + 1] < hi;
        t.guide[b] = (unsigned short)(v | (scan ? 0x8000 : 0) | (multi ? 0x4000 : 0));
    }
    return CG_OK;
}

struct Rep {
    cg_replica_desc d{};
    int N = 0, words = 0;
    Tables *tab = nullptr;
    void *d_eps = nullptr;
    unsigned *d_occ = nullptr;
    double *d_phi = nullptr;
    DevCounters *d_ctr = nullptr;
    // random sites: positions, partner lists (ascending partner) with their
    // running integer weights, 1/r and E dx, and the N x N coupling matrix
    bool random = false;
    std::vector<double> px, py, rg, redx;
    std::vector<int> roff;
    std::vector<unsigned> rj;
    std::vector<unsigned long long> rC;
    double Zmax = 0.0;
    double *d_px = nullptr, *d_py = nullptr, *d_G = nullptr;
    int *d_guide = nullptr;           // kRandomGuide ints per site
    uint2 *d_rec = nullptr;           // running weight and partner of each pair
    double2 *d_rgx = nullptr;         // 1/r and E dx of each pair
    bool pair = false;                // the handle proposes two-electron hops
    // random sites: every partner list holds at most 255 pairs, and on one
    // CTA the compacted guide records fit shared memory beside eps
    bool guide_small = false, sguide = false;
};

struct Group {
    int L = 0, first = 0, count = 0, threads = 0, smem = 0;
    int dim = 2;                     // 2: square lattice, 3: cubic lattice
    bool random = false;             // random-site replicas (pr_random)
    bool sguide = false;             // their guide records in shared memory
    int cluster = 1;                 // CTAs per replica
    unsigned M = 4096;               // labels per round when cg_run is given M = 0
    bool tuned = false;
    cudaStream_t st = nullptr;       // side stream (handles with several groups)
    cudaEvent_t done = nullptr;      // join event on that stream
    bool tc = false;                 // refresh on the tensor cores
    unsigned char *d_img = nullptr;  // S image scratch of the tensor-core refresh
    int *d_err = nullptr;            // its error word
    bool fft = false;                // refresh by the convolution theorem
    float2 *d_fft = nullptr;         // its transform buffer (a complex value per
                                     // site per replica pair)
};

// dynamic shared memory the contraction may take: the 227 KiB per-CTA opt-in
// of sm_100-class GPUs less 1 KiB for its static barriers
constexpr int kTcSmemLimit = 227 * 1024 - 1024;

// Whether a group of `count` binary32 replicas of side L and dimension dim
// refreshes on the tensor cores: the site count must be a multiple of 128 and
// the contraction's stages plus the folded table must fit one CTA's shared
// memory.
// In-place DFT (exponent -2 pi i j k / n) of n complex values at stride
// `stride`, binary64, for the refresh's host-side table: radix 2 for n = 2^m,
// the plain sum otherwise (n <= 192 there).
void host_fft(std::complex<double> *x, int n, size_t stride)
{
    if (n & (n - 1)) {
        std::vector<std::complex<double>> in(n), w(n);
        for (int j = 0; j < n; ++j) {
            in[j] = x[(size_t)j * stride];
            const double a = -2.0 * M_PI * (double)j / (double)n;
            w[j] = std::complex<double>(std::cos(a), std::sin(a));
        }
        for (int k = 0; k < n; ++k) {
            std::complex<double> acc = 0.0;
            for (int j = 0; j < n; ++j) acc += in[j] * w[(size_t)j * k % n];
            x[(size_t)k * stride] = acc;
        }
        return;
    }
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[(size_t)i * stride], x[(size_t)j * stride]);
    }
    for (int len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                std::complex<double> &a = x[(size_t)(i + k) * stride];
                std::complex<double> &b = x[(size_t)(i + k + len / 2) * stride];
                const std::complex<double> u = a, v = b * w;
                a = u + v;
                b = u - v;
            }
    }
}

// DFT(g) / N of the minimum-image 1/r on the L^dim torus (g(0) = 0), rounded
// to binary32, and the twiddles of the device transforms.
void build_fft_tables(Tables &t)
{
    const int L = t.L, H1 = t.H1;
    const size_t N = t.dim == 3 ? (size_t)L * L * L : (size_t)L * L;
    std::vector<std::complex<double>> g(N);
    const int Lz = t.dim == 3 ? L : 1;
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                const int fz = t.dim == 3 ? std::min(z, L - z) : 0;
                const int fy = std::min(y, L - y), fx = std::min(x, L - x);
                g[((size_t)z * L + y) * L + x] = t.t64[((size_t)fz * H1 + fy) * H1 + fx];
            }
    const size_t lines = N / L;
    for (size_t r = 0; r < lines; ++r) host_fft(g.data() + r * L, L, 1);          // x
    for (int z = 0; z < Lz; ++z)
        for (int x = 0; x < L; ++x) host_fft(g.data() + (size_t)z * L * L + x, L, L);   // y
    if (t.dim == 3)
        for (size_t c = 0; c < (size_t)L * L; ++c) host_fft(g.data() + c, L, (size_t)L * L);
    t.ghat.resize(N);
    for (size_t k = 0; k < N; ++k) t.ghat[k] = (float)(g[k].real() / (double)N);
    t.tw.resize(L);
    for (int k = 0; k < L; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)L;
        t.tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
}

// Whether a group of binary32 replicas of side L refreshes by the FFT:
// L = 2^m or 3 2^m (CG_REFRESH_AUTO or CG_REFRESH_FFT).
bool group_uses_fft(const cg_opts &o, int L, int dim)
{
    if (o.precision != CG_FP32 || !refresh_fft_size_ok(L)) return false;
    if (dim != 2 && dim != 3) return false;
    return o.refresh_kind == CG_REFRESH_AUTO || o.refresh_kind == CG_REFRESH_FFT;
}

bool group_uses_tc(const cg_opts &o, int L, int count, int dim)
{
    const long long N = dim == 3 ? (long long)L * L * L : (long long)L * L;
    const int H1 = L / 2 + 1, tab = dim == 3 ? H1 * H1 * H1 : H1 * H1;
    const int R_pad = (std::min(count, refresh_tc_max_replicas(dim)) + 15) / 16 * 16;
    if (o.precision != CG_FP32 || N % 128 != 0) return false;
    if (refresh_tc_smem_bytes(R_pad, tab) > kTcSmemLimit) return false;
    if (group_uses_fft(o, L, dim)) return false;
    if (o.refresh_kind == CG_REFRESH_BF16X2) return true;
    if (o.refresh_kind == CG_REFRESH_AUTO) return count >= 8;
    return false;
}

size_t tc_img_bytes(int L, int dim, int count)
{
    const int N = dim == 3 ? L * L * L : L * L;
    return refresh_tc_scratch_bytes(N, dim, std::min(count, refresh_tc_max_replicas(dim)));
}

}  // namespace

struct cg_handle {
    cg_opts opts{};
    int device = 0;
    int clock_khz = 2000000;       // peak SM clock (per-hop limit in cycles)
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<Rep> reps;
    std::vector<std::unique_ptr<Tables>> tables;
    std::vector<Group> groups;
    DevReplica *d_reps = nullptr;
    int *d_index = nullptr;
    std::vector<int> order;          // group position -> replica index (host copy of d_index)
    std::vector<DevReplica> h_reps;
    // memory: cudaMalloc'd pointers, or a caller workspace
    bool ws_mode = false;
    char *ws = nullptr;
    size_t ws_bytes = 0, ws_used = 0;
    std::vector<void *> allocs;
    // run state
    unsigned long long hops_since_refresh = 0;
    double max_err_run = 0.0;
    int toy = 0;
    double toy_A0 = 0.0;
    cg_hop *d_log = nullptr;
    bool pending = false;
    // pinned host copies of every replica's counter block (group order) and
    // of each group's refresh error word, read back in one copy per group
    // when a run is collected
    DevCounters *h_ctr = nullptr;
    int *h_err = nullptr;
    cudaEvent_t fork = nullptr;      // fork event for the groups' side streams
    cg_trace_point *d_trace = nullptr;
    int trace_cap = 0;
    // captured CUDA graphs of cg_run, keyed by (n_hops, M, hops since refresh)
    struct GraphEntry {
        unsigned long long n_hops, hsr_before, hsr_after;
        unsigned M;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
};

namespace {

int dalloc(cg_handle *h, void **p, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (h->ws_mode) {
        if (h->ws_used + bytes > h->ws_bytes)
            return fail(CG_ENOMEM, "workspace too small");
        *p = h->ws + h->ws_used;
        h->ws_used += bytes;
        return CG_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(CG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    return CG_OK;
}

// 2 for the square lattice (dim 0 or 2), 3 for the cubic lattice
int dim_of(const cg_replica_desc &d) { return d.dim == 3 ? 3 : 2; }

// sites of a replica: L^2 or L^3
int sites_of(const cg_replica_desc &d)
{
    return dim_of(d) == 3 ? d.L * d.L * d.L : d.L * d.L;
}

int check_desc(const cg_replica_desc &d)
{
    if (d.dim != 0 && d.dim != 2 && d.dim != 3) return fail(CG_EINVAL, "dim must be 0, 2 or 3");
    if (d.sites != CG_SITES_LATTICE && d.sites != CG_SITES_RANDOM)
        return fail(CG_EINVAL, "sites must be CG_SITES_LATTICE or CG_SITES_RANDOM");
    if (d.sites == CG_SITES_RANDOM && d.dim == 3)
        return fail(CG_EINVAL, "random sites live in the two-dimensional box");
    if (d.L < 4 || d.L > 1024 || (d.L & 1))
        return fail(CG_EINVAL, "L must be even and in [4, 1024]");
    if (d.dim == 3 && d.L > 64) return fail(CG_EINVAL, "a cubic lattice needs L <= 64");
    const double N = (double)sites_of(d);
    if (!(d.nu > 0.0 && d.nu < 1.0)) return fail(CG_EINVAL, "nu must be in (0, 1)");
    if (std::fabs(d.nu * N - std::floor(d.nu * N + 0.5)) > 1e-9)
        return fail(CG_EINVAL, "nu * N must be an integer");
    if (d.r_max < 1 || 2 * d.r_max >= d.L) return fail(CG_EINVAL, "need 1 <= r_max < L/2");
    if (!(d.xi > 0.0) || !std::isfinite(d.xi)) return fail(CG_EINVAL, "xi must be > 0");
    if (!(d.T > 0.0) || !std::isfinite(d.T)) return fail(CG_EINVAL, "T must be > 0");
    if (!(d.W >= 0.0) || !std::isfinite(d.W)) return fail(CG_EINVAL, "W must be >= 0");
    if (!std::isfinite(d.E)) return fail(CG_EINVAL, "E must be finite");
    // random sites keep eps (binary64) in the shared memory of one CTA or of
    // a cluster of up to 8 (227 KiB opt-in per CTA on sm_100-class GPUs,
    // 2 KiB left for the kernel's static part), and G (8 N^2 bytes) in
    // device memory: refuse before the geometry is built
    if (d.sites == CG_SITES_RANDOM &&
        (N > 131072.0 || random_smem_bytes((int)N, 8) > 227 * 1024 - 2048))
        return fail(CG_EINVAL, "random-site replicas need N <= 131072 sites (L <= 362)");
    return CG_OK;
}

// Two-electron hops: a label is a pair proposal iff its fourth Philox word
// is below this threshold, floor(pair_frac 2^32).
unsigned pair_threshold(const cg_opts &o)
{
    return o.pair_frac > 0.0 ? (unsigned)std::floor(o.pair_frac * 4294967296.0) : 0u;
}

// The total proposal rate: N Z, and with pair proposals N Z / (1 - T_p 2^-32),
// so that the single-hop attempts keep their rate.
double gamma_of(const Rep &r, const cg_opts &o)
{
    const double g = (double)r.N * (r.random ? r.Zmax : r.tab->Z);
    const unsigned Tp = pair_threshold(o);
    return Tp ? g / (1.0 - (double)Tp * 0x1p-32) : g;
}

// The single-hop cluster kernel on the cubic lattice keeps 1/r indexed by
// r^2 (3 (L/2)^2 + 1 entries) instead of the (L/2+1)^3 folded table.
int persistent_smem(const Rep &r, int precision, int cluster = 1)
{
    if (r.random) return random_smem_bytes(r.N, cluster, cluster == 1 && r.sguide);
    const int rb = precision == CG_FP64 ? 8 : 4;
    const bool r2 = dim_of(r.d) == 3 && cluster > 1 && !r.pair;
    const int ntab = r2 ? (int)r.tab->r2_64.size() : (int)r.tab->t64.size();
    return smem_layout(r.N / cluster, ntab, r.tab->V, r.words, rb).total;
}

// L must be a multiple of this for a cluster of c CTAs: c on the cubic
// lattice (whole z-planes per CTA), 2c on the square lattice (each CTA holds
// L/(2c) base rows and their partner rows y + L/2); random sites split by
// site index, any L.
int cluster_rows_unit(const cg_replica_desc &d, int c)
{
    if (d.sites == CG_SITES_RANDOM) return 2;
    return dim_of(d) == 3 ? c : 2 * c;
}

// CTAs per replica: 1 when the replica fits one CTA's shared memory, else the
// smallest cluster of 2, 4 or 8 CTAs (each holding L/C rows of eps, or L/C
// z-planes on the cubic lattice) that fits; a forced size is used when it
// fits.  0 when nothing fits.
int choose_cluster(const cg_opts &o, const Rep &r, int optin)
{
    // room for the kernels' static shared memory (the pair-hop cluster
    // kernel's exchange slots take it past 2 KiB)
    const int budget = optin - (o.pair_frac > 0.0 ? 3072 : 2048);
    if (o.cluster_size > 1) {
        const int c = o.cluster_size;
        if ((c == 2 || c == 4 || c == 8) && r.d.L % cluster_rows_unit(r.d, c) == 0 &&
            (r.random || r.d.L >= 16) && persistent_smem(r, o.precision, c) <= budget)
            return c;
        return 0;
    }
    if (persistent_smem(r, o.precision, 1) <= budget) return 1;
    for (int c = 2; c <= 8; c *= 2)
        if (r.d.L % cluster_rows_unit(r.d, c) == 0 && persistent_smem(r, o.precision, c) <= budget)
            return c;
    return 0;
}

// CTA size of a single-CTA group: the update needs at least L/2 threads (one
// per base column); 384 is accepted as given.
int choose_threads(const cg_opts &o, int L, int smem)
{
    int t = o.block_threads;
    if (t == 0) t = (o.precision == CG_FP64 || smem > 110 * 1024) ? 1024 : 512;
    while (t < L / 2 && t < 1024) t = (t == 384) ? 512 : 2 * t;
    return t;
}

unsigned magic_for(int L) { return (unsigned)(4294967296ull / (unsigned long long)L + 1ull); }

void fill_dev(const Rep &r, const cg_opts &o, DevReplica &dr, cg_hop *log)
{
    std::memset(&dr, 0, sizeof(dr));
    const Tables &t = *r.tab;
    dr.L = r.d.L; dr.N = r.N; dr.H1 = t.H1; dr.V = t.V; dr.words = r.words;
    dr.dim = t.dim;
    dr.magicL = magic_for(r.d.L);
    dr.key0 = (unsigned)r.d.seed;
    dr.key1 = (unsigned)(r.d.seed >> 32);
    dr.replica = r.d.replica;
    dr.nu = r.d.nu; dr.T = r.d.T; dr.E = r.d.E;
    dr.negC0nu = -r.d.nu * t.C0;
    dr.Gamma = gamma_of(r, o);
    dr.pair_T = pair_threshold(o);
    dr.pair_R = dr.pair_T ? o.pair_rmax : 0;
    dr.tinv64 = t.d_t64; dr.tinv32 = t.d_t32; dr.thr = t.d_thr; dr.disp = t.d_disp;
    dr.tinv_r2_64 = t.d_r2_64; dr.tinv_r2_32 = t.d_r2_32;
    dr.tinvd = t.d_tinvd;
    dr.guide = t.d_guide;
    dr.C0 = t.C0;
    dr.eps = r.d_eps; dr.occ = r.d_occ; dr.phi = r.d_phi; dr.ctr = r.d_ctr;
    dr.log = log;
    dr.G = r.d_G; dr.rguide = r.d_guide; dr.rrec = r.d_rec; dr.rgx = r.d_rgx;
    dr.rguide_small = r.guide_small ? 1 : 0;
}

// The device form of a random-site replica's partner lists: per site the
// kRandomGuide record (list bounds, the pair each x1 bucket starts at, the
// last running weight), per pair (C mod 2^32, j | (C >> 32) << 31) and
// (1/r, E dx).
void pack_random(const Rep &r, std::vector<int> &guide, std::vector<uint32_t> &rec,
                 std::vector<double> &rgx)
{
    const int N = r.N;
    const size_t m = r.rj.size();
    guide.assign((size_t)N * kRandomGuide, 0);
    rec.assign(2 * m, 0u);
    rgx.assign(2 * m, 0.0);
    for (size_t k = 0; k < m; ++k) {
        // C_k <= 2^32 in 33 bits: the low word, and its top bit above the
        // partner (partners < N < 2^31)
        rec[2 * k] = (uint32_t)r.rC[k];
        rec[2 * k + 1] = r.rj[k] | ((uint32_t)(r.rC[k] >> 32) << 31);
        rgx[2 * k] = r.rg[k];
        rgx[2 * k + 1] = r.redx[k];
    }
    for (int s = 0; s < N; ++s) {
        int *g = guide.data() + (size_t)s * kRandomGuide;
        const int lo = r.roff[s], hi = r.roff[s + 1];
        g[0] = lo;
        g[1] = hi;
        int a = lo;
        for (int b = 0; b < kRandomBuckets; ++b) {
            const unsigned long long v = (unsigned long long)b << (32 - 4);
            while (a < hi && !(v < r.rC[a])) ++a;      // smallest a with v < C_a
            const int start = a < hi ? a : (hi > lo ? hi - 1 : lo);
            const uint32_t off = (uint32_t)(start - lo);   // < 2^16: lists hold < N pairs
            uint32_t &w = reinterpret_cast<uint32_t &>(g[4 + b / 2]);
            w |= (b & 1) ? (off << 16) : off;
        }
        const unsigned long long last = hi > lo ? r.rC[hi - 1] : 0ull;
        g[2] = (int)(uint32_t)last;
        g[3] = (int)(uint32_t)(last >> 32);
    }
}

// Random sites: positions from Philox counter (s, 3, 0xFFFFFFFF, replica),
// x = L (x0 + 1/2) 2^-32 and y = L (x1 + 1/2) 2^-32; the partners of s are
// the t != s with r_st <= r_max (minimum image), in ascending t; weight
// w = exp(-2 r / xi), Zmax the largest per-site sum, integer weights
// floor(2^32 w / Zmax) (at most 2^32 - 1) and their running sums per list.
// Coincident sites are refused.
int build_random(Rep &r)
{
    const int L = r.d.L, N = r.N, R = r.d.r_max;
    const uint32_t k0 = (uint32_t)r.d.seed, k1 = (uint32_t)(r.d.seed >> 32);
    const double Ld = (double)L;
    r.px.resize(N);
    r.py.resize(N);
    for (int s = 0; s < N; ++s) {
        uint32_t x[4];
        philox4x32_10((uint32_t)s, 3u, 0xFFFFFFFFu, r.d.replica, k0, k1, x);
        r.px[s] = Ld * (((double)x[0] + 0.5) * 0x1p-32);
        r.py[s] = Ld * (((double)x[1] + 0.5) * 0x1p-32);
    }
    auto mi = [&](double d) {
        if (d > 0.5 * Ld) return d - Ld;
        if (d < -0.5 * Ld) return d + Ld;
        return d;
    };
    // candidate partners from a cell list: nc x nc cells of side L/nc >= R + 1,
    // so every t within r_max of s lies in the 3 x 3 cells around s's (the
    // margin of 1 covers the rounding of the cell index); the candidates are
    // taken in ascending t, the order of the definition, so Z sums in the
    // same order.  With fewer than 3 cells per axis every t is a candidate.
    const int nc = L / (R + 1) >= 3 ? L / (R + 1) : 1;
    auto cell_of = [&](double v) {
        int c = (int)std::floor(v * (double)nc / Ld);
        return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
    };
    std::vector<int> cstart((size_t)nc * nc + 1, 0), cell(N), members(N);
    for (int s = 0; s < N; ++s) {
        cell[s] = cell_of(r.py[s]) * nc + cell_of(r.px[s]);
        ++cstart[cell[s] + 1];
    }
    for (int c = 0; c < nc * nc; ++c) cstart[c + 1] += cstart[c];
    {
        std::vector<int> fill(cstart.begin(), cstart.end() - 1);
        for (int s = 0; s < N; ++s) members[fill[cell[s]]++] = s;   // ascending s per cell
    }
    r.roff.assign(N + 1, 0);
    r.rj.clear(); r.rg.clear(); r.redx.clear(); r.rC.clear();
    std::vector<double> w, Z(N, 0.0), dxs;
    std::vector<int> cand;
    for (int s = 0; s < N; ++s) {
        r.roff[s] = (int)r.rj.size();
        cand.clear();
        if (nc == 1) {
            for (int t = 0; t < N; ++t) cand.push_back(t);
        } else {
            const int cx = cell[s] % nc, cy = cell[s] / nc;
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    const int c = ((cy + oy + nc) % nc) * nc + (cx + ox + nc) % nc;
                    cand.insert(cand.end(), members.begin() + cstart[c],
                                members.begin() + cstart[c + 1]);
                }
            std::sort(cand.begin(), cand.end());
        }
        for (const int t : cand) {
            if (t == s) continue;
            const double dx = mi(r.px[t] - r.px[s]);
            const double dy = mi(r.py[t] - r.py[s]);
            const double rr = std::sqrt(dx * dx + dy * dy);
            if (rr == 0.0) return fail(CG_EINVAL, "random sites: two sites coincide");
            if (rr > (double)R) continue;
            r.rj.push_back((unsigned)t);
            r.rg.push_back(1.0 / rr);
            dxs.push_back(dx);
            const double ws = host_exp(-2.0 * rr / r.d.xi);
            w.push_back(ws);
            Z[s] = Z[s] + ws;
        }
        if ((int)r.rj.size() - r.roff[s] >= 65536)
            return fail(CG_EINVAL, "random sites: a partner list holds 2^16 or more pairs "
                                   "(r_max too large)");
    }
    r.roff[N] = (int)r.rj.size();
    r.Zmax = 0.0;
    for (int s = 0; s < N; ++s) if (Z[s] > r.Zmax) r.Zmax = Z[s];
    if (!(r.Zmax > 0.0)) return fail(CG_EINVAL, "random sites: no site has a partner within r_max");
    r.rC.resize(r.rj.size());
    r.redx.resize(r.rj.size());
    for (int s = 0; s < N; ++s) {
        unsigned long long run = 0;
        for (int m = r.roff[s]; m < r.roff[s + 1]; ++m) {
            unsigned long long Wm = (unsigned long long)std::floor((w[m] / r.Zmax) * 4294967296.0);
            if (Wm > 0xFFFFFFFFull) Wm = 0xFFFFFFFFull;
            run += Wm;
            r.rC[m] = run;
            r.redx[m] = r.d.E * dxs[m];
        }
    }
    return CG_OK;
}

void host_setup_state(const cg_replica_desc &d, std::vector<double> &phi,
                      std::vector<unsigned char> &n)
{
    const int N = sites_of(d);
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    phi.resize(N);
    n.assign(N, 0);
    std::vector<std::pair<uint32_t, uint32_t>> keys(N);
    for (int s = 0; s < N; ++s) {
        uint32_t x[4];
        philox4x32_10((uint32_t)s, 1u, 0xFFFFFFFFu, d.replica, k0, k1, x);
        const double u = ((double)x[0] + 0.5) * 0x1p-32;
        phi[s] = d.W * (u - 0.5);
        philox4x32_10((uint32_t)s, 2u, 0xFFFFFFFFu, d.replica, k0, k1, x);
        keys[s] = {x[0], (uint32_t)s};
    }
    std::sort(keys.begin(), keys.end());
    const int nocc = (int)std::floor(d.nu * N + 0.5);
    for (int s = 0; s < nocc; ++s) n[keys[s].second] = 1;
}

std::vector<unsigned> pack_bits(const unsigned char *n, int N)
{
    std::vector<unsigned> w((N + 31) / 32, 0u);
    for (int s = 0; s < N; ++s)
        if (n[s]) w[s >> 5] |= 1u << (s & 31);
    return w;
}

int replica_index_ok(const cg_handle *h, int r)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (r < 0 || r >= (int)h->reps.size()) return fail(CG_EINVAL, "replica out of range");
    return CG_OK;
}

// Energy of Eq. 1 (field term with x in [0, L)) from eps:
// H = sum n phi + 1/2 sum (n - nu)(eps - phi) - E sum n x.
double energy_from_eps(const cg_replica_desc &d, const unsigned char *n, const double *eps,
                       const double *phi, long long *P_out, const double *px = nullptr)
{
    const int N = sites_of(d);
    double h1 = 0.0, h2 = 0.0, X = 0.0;
    long long P = 0;
    for (int s = 0; s < N; ++s) {
        h1 += n[s] ? phi[s] : 0.0;
        h2 += ((double)n[s] - d.nu) * (eps[s] - phi[s]);
        if (n[s]) P += s % d.L;
        if (n[s] && px) X += px[s];
    }
    if (px) {
        // random sites: the field term with the real x; no dipole counter
        *P_out = 0;
        return h1 + 0.5 * h2 - d.E * X;
    }
    *P_out = P;
    return h1 + 0.5 * h2 - d.E * (double)P;
}

int read_eps_host(cg_handle *h, const Rep &r, double *out)
{
    if (h->opts.precision == CG_FP64) {
        CG_CUDA(cudaMemcpyAsync(out, r.d_eps, sizeof(double) * r.N, cudaMemcpyDeviceToHost, h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
    } else {
        std::vector<float> f(r.N);
        CG_CUDA(cudaMemcpyAsync(f.data(), r.d_eps, sizeof(float) * r.N, cudaMemcpyDeviceToHost,
                                h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
        for (int s = 0; s < r.N; ++s) out[s] = (double)f[s];
    }
    return CG_OK;
}

// Upload occupation (+phi), rebuild or set eps, set or recompute counters.
int load_state(cg_handle *h, int ri, const unsigned char *n, const double *eps,
               const double *phi, const cg_counters *c)
{
    Rep &r = h->reps[ri];
    const std::vector<unsigned> words = pack_bits(n, r.N);
    CG_CUDA(cudaMemcpyAsync(r.d_occ, words.data(), 4 * words.size(), cudaMemcpyHostToDevice, h->st));
    if (phi)
        CG_CUDA(cudaMemcpyAsync(r.d_phi, phi, sizeof(double) * r.N, cudaMemcpyHostToDevice, h->st));
    if (eps) {
        if (h->opts.precision == CG_FP64) {
            CG_CUDA(cudaMemcpyAsync(r.d_eps, eps, sizeof(double) * r.N, cudaMemcpyHostToDevice,
                                    h->st));
        } else {
            std::vector<float> f(r.N);
            for (int s = 0; s < r.N; ++s) f[s] = (float)eps[s];
            CG_CUDA(cudaMemcpyAsync(r.d_eps, f.data(), sizeof(float) * r.N, cudaMemcpyHostToDevice,
                                    h->st));
            CG_CUDA(cudaStreamSynchronize(h->st));
        }
    } else if (r.random) {
        CG_CUDA(launch_eps_init_random(h->d_reps + ri, r.N, h->st));
    } else {
        CG_CUDA(launch_eps_init(h->d_reps + ri, r.N, (int)r.tab->t64.size(), r.words,
                                h->opts.precision, h->st));
    }
    DevCounters dc;
    std::memset(&dc, 0, sizeof(dc));
    if (c) {
        dc.rounds = c->rounds; dc.hops = c->hops; dc.attempts = c->attempts;
        dc.evaluated = c->evaluated; dc.P = c->P; dc.energy = c->energy;
        dc.time = c->time;
    } else {
        std::vector<double> e(r.N), ph(r.N);
        int rc = read_eps_host(h, r, e.data());
        if (rc) return rc;
        CG_CUDA(cudaMemcpyAsync(ph.data(), r.d_phi, sizeof(double) * r.N, cudaMemcpyDeviceToHost,
                                h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
        long long P = 0;
        dc.energy = energy_from_eps(r.d, n, e.data(), ph.data(), &P,
                                    r.random ? r.px.data() : nullptr);
        dc.P = P;
    }
    CG_CUDA(cudaMemcpyAsync(r.d_ctr, &dc, sizeof(dc), cudaMemcpyHostToDevice, h->st));
    CG_CUDA(cudaStreamSynchronize(h->st));
    return CG_OK;
}

size_t plan_bytes(int R, const cg_replica_desc *reps, const cg_opts &o)
{
    // mirrors the allocations of create_impl (each rounded up to 256 bytes)
    const int precision = o.precision;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    std::vector<std::tuple<int, int, int>> groups;   // (L, dim, count)
    for (int k = 0; k < R; ++k) {
        bool found = false;
        for (auto &g : groups)
            if (std::get<0>(g) == reps[k].L && std::get<1>(g) == dim_of(reps[k])) {
                ++std::get<2>(g);
                found = true;
            }
        if (!found) groups.push_back({reps[k].L, dim_of(reps[k]), 1});
    }
    size_t tc_total = 0;
    for (auto &g : groups)
        if (group_uses_fft(o, std::get<0>(g), std::get<1>(g))) {
            const size_t L = (size_t)std::get<0>(g);
            const size_t N = std::get<1>(g) == 3 ? L * L * L : L * L;
            tc_total += up(refresh_fft_buffer_bytes((int)N, std::get<2>(g))) + up(N * 4) +
                        up(L * 8);
        }
    for (auto &g : groups)
        if (group_uses_tc(o, std::get<0>(g), std::get<2>(g), std::get<1>(g)))
            tc_total += up(tc_img_bytes(std::get<0>(g), std::get<1>(g), std::get<2>(g))) +
                        up(sizeof(int));
    size_t total = up(sizeof(DevReplica) * (size_t)R) + up(sizeof(int) * (size_t)R);
    std::vector<std::tuple<int, int, double, int>> seen;
    for (int k = 0; k < R; ++k) {
        const cg_replica_desc &d = reps[k];
        const size_t N = (size_t)sites_of(d), words = (N + 31) / 32;
        total += up(N * (precision == CG_FP64 ? 8 : 4)) + up(words * 4) + up(N * 8) +
                 up(sizeof(DevCounters));
        if (d.sites == CG_SITES_RANDOM) {
            // positions, G, and the partner lists (their length needs the
            // geometry itself)
            Rep tmp;
            tmp.d = d;
            tmp.N = (int)N;
            const size_t cnt = build_random(tmp) == CG_OK ? tmp.rj.size() : 0;
            const size_t c1 = cnt ? cnt : 1;
            total += 2 * up(N * 8) + up(N * N * 8) + up(N * kRandomGuide * 4) + up(c1 * 8) + up(c1 * 16);
        }
        auto key = std::make_tuple(d.L, d.r_max, d.xi, dim_of(d));
        if (std::find(seen.begin(), seen.end(), key) == seen.end()) {
            seen.push_back(key);
            const size_t H1 = d.L / 2 + 1;
            const size_t tab = dim_of(d) == 3 ? H1 * H1 * H1 : H1 * H1;
            const int Rz = dim_of(d) == 3 ? d.r_max : 0;
            size_t V = 0;
            for (int dz = -Rz; dz <= Rz; ++dz)
                for (int dy = -d.r_max; dy <= d.r_max; ++dy)
                    for (int dx = -d.r_max; dx <= d.r_max; ++dx) {
                        const int r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 > 0 && r2 <= d.r_max * d.r_max) ++V;
                    }
            total += up(tab * 8) + up(tab * 4) + up(V * 4) + up(V * 4) + up(V * 8) +
                     up((size_t)kGuide * 2) + up(tab * 4);
            if (dim_of(d) == 3) {
                const size_t n2 = 3 * (size_t)(d.L / 2) * (d.L / 2) + 1;
                total += up(n2 * 8) + up(n2 * 4);
            }
        }
    }
    return total + tc_total;
}

cg_handle *create_impl(int R, const cg_replica_desc *reps, const cg_opts *opts, void *ws,
                       size_t ws_bytes)
{
    if (R <= 0 || !reps) { fail(CG_EINVAL, "need R >= 1 replica descriptors"); return nullptr; }
    cg_opts o{};
    if (opts) o = *opts;
    if (o.precision != CG_FP64 && o.precision != CG_FP32) {
        fail(CG_EINVAL, "precision must be CG_FP64 or CG_FP32");
        return nullptr;
    }
    if (o.block_threads && (o.block_threads != 256 && o.block_threads != 384 &&
                            o.block_threads != 512 && o.block_threads != 1024)) {
        fail(CG_EINVAL, "block_threads must be 0, 256, 384, 512 or 1024");
        return nullptr;
    }
    if (o.refresh_kind < CG_REFRESH_AUTO || o.refresh_kind > CG_REFRESH_FFT) {
        fail(CG_EINVAL, "refresh_kind must be CG_REFRESH_AUTO, _FP64, _BF16X2 or _FFT");
        return nullptr;
    }
    if (o.time_mode != CG_TIME_DETERMINISTIC && o.time_mode != CG_TIME_GAUSSIAN) {
        fail(CG_EINVAL, "time_mode must be CG_TIME_DETERMINISTIC or CG_TIME_GAUSSIAN");
        return nullptr;
    }
    if (o.max_rounds_per_hop == 0) o.max_rounds_per_hop = 1ull << 32;
    for (int k = 0; k < R; ++k)
        if (check_desc(reps[k]) != CG_OK) return nullptr;
    if (!(o.pair_frac >= 0.0 && o.pair_frac < 1.0)) {
        fail(CG_EINVAL, "pair_frac must be in [0, 1)");
        return nullptr;
    }
    for (int k = 0; k < R; ++k)
        if (reps[k].sites == CG_SITES_RANDOM &&
            (o.precision != CG_FP64 || o.pair_frac > 0.0 || o.time_mode != CG_TIME_DETERMINISTIC)) {
            fail(CG_EINVAL, "random sites run in binary64, single hops and deterministic time");
            return nullptr;
        }
    if (o.pair_frac > 0.0) {
        for (int k = 0; k < R; ++k)
            if (o.pair_rmax < 1 || 2 * o.pair_rmax >= reps[k].L) {
                fail(CG_EINVAL, "two-electron hops need 1 <= pair_rmax < L/2");
                return nullptr;
            }
    }

    std::unique_ptr<cg_handle> h(new cg_handle());
    h->opts = o;
    h->device = o.device;
    if (cudaSetDevice(o.device) != cudaSuccess) {
        fail(CG_ECUDA, "cudaSetDevice failed");
        return nullptr;
    }
    {
        int khz = 0;
        if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, o.device) == cudaSuccess && khz > 0)
            h->clock_khz = khz;
    }
    if (ws) {
        if (((uintptr_t)ws & 255) != 0) { fail(CG_EINVAL, "workspace must be 256-byte aligned"); return nullptr; }
        h->ws_mode = true;
        h->ws = (char *)ws;
        h->ws_bytes = ws_bytes;
    }
    if (o.stream) {
        h->st = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
            fail(CG_ECUDA, "cudaStreamCreate failed");
            return nullptr;
        }
        h->own_stream = true;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, o.device);

    auto destroy_partial = [&]() { cg_destroy(h.release()); };

    // tables, shared by replicas of equal (L, r_max, xi)
    h->reps.resize(R);
    for (int k = 0; k < R; ++k) {
        Rep &r = h->reps[k];
        r.d = reps[k];
        r.N = sites_of(r.d);
        r.words = (r.N + 31) / 32;
        r.random = r.d.sites == CG_SITES_RANDOM;
        r.pair = o.pair_frac > 0.0;
        if (r.random && build_random(r) != CG_OK) {
            destroy_partial();
            return nullptr;
        }
        if (r.random) {
            int longest = 0;
            for (int k = 0; k < r.N; ++k) longest = std::max(longest, r.roff[k + 1] - r.roff[k]);
            r.guide_small = longest <= 255;
            r.sguide = r.guide_small && random_smem_bytes(r.N, 1, true) <= optin - 2048;
        }
        for (auto &t : h->tables)
            if (t->L == r.d.L && t->r_max == r.d.r_max && t->xi == r.d.xi && t->dim == dim_of(r.d))
                r.tab = t.get();
        if (!r.tab) {
            std::unique_ptr<Tables> t(new Tables());
            if (build_tables(*t, r.d.L, r.d.xi, r.d.r_max, dim_of(r.d)) != CG_OK) {
                destroy_partial();
                return nullptr;
            }
            if (!r.random && group_uses_fft(o, r.d.L, dim_of(r.d))) build_fft_tables(*t);
            r.tab = t.get();
            h->tables.push_back(std::move(t));
        }
        if (choose_cluster(o, r, optin) == 0) {
            fail(CG_EINVAL, "replica does not fit the shared memory of one CTA or of a "
                            "cluster of up to 8 CTAs (or the forced cluster size does not "
                            "fit, or L is not a multiple of twice it on the square lattice)");
            destroy_partial();
            return nullptr;
        }
    }
    // device memory
    if (dalloc(h.get(), (void **)&h->d_reps, sizeof(DevReplica) * R) ||
        dalloc(h.get(), (void **)&h->d_index, sizeof(int) * R)) { destroy_partial(); return nullptr; }
    for (auto &t : h->tables) {
        if (dalloc(h.get(), (void **)&t->d_t64, t->t64.size() * 8) ||
            dalloc(h.get(), (void **)&t->d_t32, t->t32.size() * 4) ||
            dalloc(h.get(), (void **)&t->d_thr, t->thr.size() * 4) ||
            dalloc(h.get(), (void **)&t->d_disp, t->disp.size() * 4) ||
            dalloc(h.get(), (void **)&t->d_tinvd, t->tinvd.size() * 8) ||
            dalloc(h.get(), (void **)&t->d_guide, t->guide.size() * 2) ||
            dalloc(h.get(), (void **)&t->d_split, t->split.size() * 4)) { destroy_partial(); return nullptr; }
        if (!t->ghat.empty()) {
            if (dalloc(h.get(), (void **)&t->d_ghat, t->ghat.size() * 4) ||
                dalloc(h.get(), (void **)&t->d_tw, t->tw.size() * 8)) { destroy_partial(); return nullptr; }
            cudaMemcpyAsync(t->d_ghat, t->ghat.data(), t->ghat.size() * 4, cudaMemcpyHostToDevice, h->st);
            cudaMemcpyAsync(t->d_tw, t->tw.data(), t->tw.size() * 8, cudaMemcpyHostToDevice, h->st);
        }
        if (t->dim == 3) {
            if (dalloc(h.get(), (void **)&t->d_r2_64, t->r2_64.size() * 8) ||
                dalloc(h.get(), (void **)&t->d_r2_32, t->r2_32.size() * 4)) { destroy_partial(); return nullptr; }
            cudaMemcpyAsync(t->d_r2_64, t->r2_64.data(), t->r2_64.size() * 8, cudaMemcpyHostToDevice, h->st);
            cudaMemcpyAsync(t->d_r2_32, t->r2_32.data(), t->r2_32.size() * 4, cudaMemcpyHostToDevice, h->st);
        }
        cudaMemcpyAsync(t->d_split, t->split.data(), t->split.size() * 4, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(t->d_t64, t->t64.data(), t->t64.size() * 8, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(t->d_t32, t->t32.data(), t->t32.size() * 4, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(t->d_thr, t->thr.data(), t->thr.size() * 4, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(t->d_disp, t->disp.data(), t->disp.size() * 4, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(t->d_tinvd, t->tinvd.data(), t->tinvd.size() * 8, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(t->d_guide, t->guide.data(), t->guide.size() * 2, cudaMemcpyHostToDevice, h->st);
    }
    for (Rep &r : h->reps) {
        if (!r.random) continue;
        const size_t N = (size_t)r.N, cnt = std::max<size_t>(r.rj.size(), 1);
        if (dalloc(h.get(), (void **)&r.d_px, N * 8) || dalloc(h.get(), (void **)&r.d_py, N * 8) ||
            dalloc(h.get(), (void **)&r.d_G, N * N * 8) ||
            dalloc(h.get(), (void **)&r.d_guide, N * kRandomGuide * 4) ||
            dalloc(h.get(), (void **)&r.d_rec, cnt * 8) ||
            dalloc(h.get(), (void **)&r.d_rgx, cnt * 16)) { destroy_partial(); return nullptr; }
        const size_t m = r.rj.size();
        std::vector<int> guide;
        std::vector<uint32_t> rec;
        std::vector<double> rgx;
        pack_random(r, guide, rec, rgx);
        cudaMemcpyAsync(r.d_px, r.px.data(), N * 8, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(r.d_py, r.py.data(), N * 8, cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(r.d_guide, guide.data(), N * kRandomGuide * 4, cudaMemcpyHostToDevice,
                        h->st);
        if (m) {
            cudaMemcpyAsync(r.d_rec, rec.data(), m * 8, cudaMemcpyHostToDevice, h->st);
            cudaMemcpyAsync(r.d_rgx, rgx.data(), m * 16, cudaMemcpyHostToDevice, h->st);
        }
        if (launch_g_build(r.d_px, r.d_py, r.d.L, r.N, r.d_G, h->st) != cudaSuccess) {
            fail(CG_ECUDA, "coupling-matrix build failed to launch");
            destroy_partial();
            return nullptr;
        }
        // the host copies served the uploads (pageable: wait before they go)
        if (cudaStreamSynchronize(h->st) != cudaSuccess) {
            fail(CG_ECUDA, "random-site geometry upload failed");
            destroy_partial();
            return nullptr;
        }
    }
    const int rb = o.precision == CG_FP64 ? 8 : 4;
    // groups of equal (sites kind, dimension, L) (one launch each), replica
    // order kept inside a group
    auto gkey = [&](int k) {
        return (h->reps[k].random ? 1 << 20 : 0) + dim_of(h->reps[k].d) * 4096 + h->reps[k].d.L;
    };
    std::vector<int> order(R);
    for (int k = 0; k < R; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gkey(a) < gkey(b); });
    // each group's eps, bitmasks, phi and counters are one block per array in
    // group order, so a group's state moves between host and device in one
    // copy per array (cg_read_group_state / cg_write_group_state)
    for (int k = 0; k < R;) {
        int e = k;
        while (e < R && gkey(order[e]) == gkey(order[k])) ++e;
        const Rep &r0 = h->reps[order[k]];
        const size_t cnt = (size_t)(e - k);
        char *eb = nullptr, *pb = nullptr;
        unsigned *ob = nullptr;
        DevCounters *cb = nullptr;
        if (dalloc(h.get(), (void **)&eb, cnt * r0.N * rb) ||
            dalloc(h.get(), (void **)&ob, cnt * r0.words * 4) ||
            dalloc(h.get(), (void **)&pb, cnt * r0.N * 8) ||
            dalloc(h.get(), (void **)&cb, cnt * sizeof(DevCounters))) { destroy_partial(); return nullptr; }
        for (int m = k; m < e; ++m) {
            Rep &r = h->reps[order[m]];
            const size_t i = (size_t)(m - k);
            r.d_eps = eb + i * r0.N * rb;
            r.d_occ = ob + i * r0.words;
            r.d_phi = reinterpret_cast<double *>(pb) + i * r0.N;
            r.d_ctr = cb + i;
        }
        k = e;
    }
    for (int k = 0; k < R;) {
        Group g;
        g.L = h->reps[order[k]].d.L;
        g.dim = dim_of(h->reps[order[k]].d);
        g.random = h->reps[order[k]].random;
        g.sguide = g.random;
        for (int m = k; m < R && gkey(order[m]) == gkey(order[k]); ++m)
            g.sguide = g.sguide && h->reps[order[m]].sguide;
        g.first = k;
        const int key = gkey(order[k]);
        int smem = 0, cluster = 1;
        for (int m = k; m < R && gkey(order[m]) == key; ++m)
            cluster = std::max(cluster, choose_cluster(o, h->reps[order[m]], optin));
        while (k < R && gkey(order[k]) == key) {
            smem = std::max(smem, persistent_smem(h->reps[order[k]], o.precision, cluster));
            ++k;
        }
        g.count = k - g.first;
        g.smem = smem;
        g.cluster = cluster;
        g.threads = choose_threads(o, g.L, smem);
        if (cluster > 1 && g.random) {
            // the random-site cluster kernel takes 256, 512 or 1024 threads
            if (g.threads == 384) g.threads = 512;
        } else if (cluster > 1) {
            // the cluster kernel maps a thread to a column: at least L threads
            if (g.threads < 512) g.threads = 512;
            while (g.threads < g.L && g.threads < 1024) g.threads *= 2;
        }
        g.fft = !g.random && group_uses_fft(o, g.L, g.dim);
        if (g.fft && dalloc(h.get(), (void **)&g.d_fft,
                            refresh_fft_buffer_bytes(dim_of(h->reps[order[g.first]].d) == 3
                                                         ? g.L * g.L * g.L : g.L * g.L,
                                                     g.count))) {
            destroy_partial();
            return nullptr;
        }
        g.tc = group_uses_tc(o, g.L, g.count, g.dim);
        if (g.tc && (dalloc(h.get(), (void **)&g.d_img, tc_img_bytes(g.L, g.dim, g.count)) ||
                     dalloc(h.get(), (void **)&g.d_err, sizeof(int)))) {
            destroy_partial();
            return nullptr;
        }
        if (g.tc) cudaMemsetAsync(g.d_err, 0, sizeof(int), h->st);
        h->groups.push_back(g);
    }
    if (h->groups.size() > 1) {
        // one stream per lattice size, forked from and joined to the handle's
        if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) {
            fail(CG_ECUDA, "cudaEventCreate failed");
            destroy_partial();
            return nullptr;
        }
        for (Group &g : h->groups)
            if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess) {
                fail(CG_ECUDA, "side stream creation failed");
                destroy_partial();
                return nullptr;
            }
    }
    h->order = order;
    h->h_reps.resize(R);
    for (int k = 0; k < R; ++k) fill_dev(h->reps[k], o, h->h_reps[k], nullptr);
    if (cudaMemcpyAsync(h->d_reps, h->h_reps.data(), sizeof(DevReplica) * R,
                        cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
        cudaMemcpyAsync(h->d_index, order.data(), sizeof(int) * R, cudaMemcpyHostToDevice,
                        h->st) != cudaSuccess) {
        fail(CG_ECUDA, "upload of replica descriptors failed");
        destroy_partial();
        return nullptr;
    }
    if (set_pr_smem_limit(o.precision, optin - 2048) != cudaSuccess ||
        set_pr_random_smem_limit(optin - 2048) != cudaSuccess) {
        fail(CG_ECUDA, "cudaFuncSetAttribute(max dynamic shared memory) failed");
        destroy_partial();
        return nullptr;
    }
    // disorder, initial occupation, eps from scratch, energy
    for (int k = 0; k < R; ++k) {
        std::vector<double> phi;
        std::vector<unsigned char> n;
        host_setup_state(h->reps[k].d, phi, n);
        if (load_state(h.get(), k, n.data(), nullptr, phi.data(), nullptr) != CG_OK) {
            destroy_partial();
            return nullptr;
        }
    }
    if (cudaStreamSynchronize(h->st) != cudaSuccess) {
        fail(CG_ECUDA, "set-up kernels failed");
        destroy_partial();
        return nullptr;
    }
    if (cudaMallocHost((void **)&h->h_ctr, sizeof(DevCounters) * (size_t)R) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_err, sizeof(int) * h->groups.size()) != cudaSuccess) {
        fail(CG_ECUDA, "pinned host buffers could not be allocated");
        destroy_partial();
        return nullptr;
    }
    return h.release();
}

// Rebuild eps of one group's replicas from scratch (binary64: the serial-order
// kernel; binary32: the tensor-core contraction or the binary64 direct sum).
int refresh_group(cg_handle *h, const Group &g, cudaStream_t st)
{
    if (h->opts.precision != CG_FP32) {
        for (int k = g.first; k < g.first + g.count; ++k) {
            const int ri = h->order[k];
            const Rep &r = h->reps[ri];
            if (r.random) {
                CG_CUDA(launch_eps_init_random(h->d_reps + ri, r.N, st));
                continue;
            }
            CG_CUDA(launch_eps_init(h->d_reps + ri, r.N, (int)r.tab->t64.size(), r.words, CG_FP64,
                                    st));
        }
        return CG_OK;
    }
    CG_CUDA(launch_reset_refresh_err(h->d_reps, h->d_index + g.first, g.count, st));
    if (g.fft) {
        const Tables &t = *h->reps[h->order[g.first]].tab;
        CG_CUDA(launch_refresh_fft(h->d_reps, h->d_index + g.first, g.count, g.L, g.dim, t.d_ghat,
                                   t.d_tw, g.d_fft, st));
    } else if (g.tc) {
        const uint32_t *split = h->reps[h->order[g.first]].tab->d_split;
        const int per = refresh_tc_max_replicas(g.dim);
        for (int c0 = 0; c0 < g.count; c0 += per) {
            const int n = std::min(per, g.count - c0);
            CG_CUDA(launch_refresh_tc(h->d_reps, h->d_index + g.first + c0, n, g.L, g.dim, split,
                                      g.d_img, g.d_err, st));
        }
    } else {
        for (int k = g.first; k < g.first + g.count; ++k) {
            const int ri = h->order[k];
            const Rep &r = h->reps[ri];
            CG_CUDA(launch_refresh_fp64(h->d_reps + ri, r.N, (int)r.tab->t64.size(), r.words, st));
        }
    }
    return CG_OK;
}

int refresh_all(cg_handle *h)
{
    for (const Group &g : h->groups) {
        const int rc = refresh_group(h, g, h->st);
        if (rc) return rc;
    }
    return CG_OK;
}

int launch_group(cg_handle *h, const Group &g, unsigned long long hops, unsigned M,
                 unsigned long long log_off, cudaStream_t st)
{
    RunArgs a{};
    a.n_hops = hops;
    a.M = M ? M : g.M;
    a.max_rounds = h->opts.max_rounds_per_hop;
    a.log_offset = log_off;
    a.hop_timeout_ns = 1000000ull * (h->opts.hop_timeout_ms ? h->opts.hop_timeout_ms : 10000u);
    // the same limit in SM cycles at the peak clock (a lower clock only makes
    // the limit longer in seconds)
    a.hop_timeout_cyc = (unsigned long long)(h->opts.hop_timeout_ms ? h->opts.hop_timeout_ms : 10000u) *
                        (unsigned long long)h->clock_khz;
    a.toy = h->toy;
    a.toy_A0 = h->toy_A0;
    a.time_mode = h->opts.time_mode;
    a.pair = h->opts.pair_frac > 0.0 ? 1 : 0;
    a.smem_guide = (g.random && g.cluster == 1 && g.sguide) ? 1 : 0;
    if (g.random && g.cluster > 1)
        CG_CUDA(launch_pr_random_cluster(h->d_reps, h->d_index + g.first, g.count, g.cluster,
                                         g.threads, g.smem, a, st));
    else if (g.random)
        CG_CUDA(launch_pr_random(h->d_reps, h->d_index + g.first, g.count, g.threads, g.smem, a,
                                 st));
    else if (g.cluster > 1)
        CG_CUDA(launch_pr_cluster(h->opts.precision, h->d_reps, h->d_index + g.first, g.count,
                                  g.cluster, g.threads, g.smem, a, st, g.L, g.dim));
    else
        CG_CUDA(launch_pr_persistent(h->opts.precision, h->d_reps, h->d_index + g.first,
                                     g.count, g.threads, g.smem, a, st, g.L, g.dim));
    return CG_OK;
}

// Queue n_hops hops of every replica: segments that end where a binary32
// refresh falls due; with several lattice sizes each group runs its segment
// (and its refresh) on its own stream between a fork and a join, so the
// groups' persistent launches overlap.
int enqueue_run(cg_handle *h, unsigned long long n_hops, unsigned M, bool logged)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (M > (1u << 24)) return fail(CG_EINVAL, "M must be in [1, 2^24] (0: per-group M)");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    const bool refresh = h->opts.precision == CG_FP32 && h->opts.refresh_every > 0;
    const bool forked = h->groups.size() > 1;
    unsigned long long done = 0;
    while (done < n_hops) {
        unsigned long long seg = n_hops - done;
        if (refresh) seg = std::min(seg, h->opts.refresh_every - h->hops_since_refresh);
        const bool refresh_now = refresh && h->hops_since_refresh + seg == h->opts.refresh_every;
        if (forked) CG_CUDA(cudaEventRecord(h->fork, h->st));
        for (const Group &g : h->groups) {
            cudaStream_t st = forked ? g.st : h->st;
            if (forked) CG_CUDA(cudaStreamWaitEvent(st, h->fork, 0));
            int rc = launch_group(h, g, seg, M, logged ? done : 0, st);
            if (!rc && refresh_now) rc = refresh_group(h, g, st);
            if (rc) return rc;
            if (forked) {
                CG_CUDA(cudaEventRecord(g.done, st));
                CG_CUDA(cudaStreamWaitEvent(h->st, g.done, 0));
            }
        }
        done += seg;
        if (refresh) h->hops_since_refresh = refresh_now ? 0 : h->hops_since_refresh + seg;
    }
    h->pending = true;
    return CG_OK;
}

// cg_run through a CUDA graph: the launches of one (n_hops, M, refresh phase)
// are captured once and replayed.
int enqueue_run_graph(cg_handle *h, unsigned long long n_hops, unsigned M)
{
    if (M > (1u << 24)) return fail(CG_EINVAL, "M must be in [1, 2^24] (0: per-group M)");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    for (const auto &e : h->graphs)
        if (e.n_hops == n_hops && e.M == M && e.hsr_before == h->hops_since_refresh) {
            CG_CUDA(cudaGraphLaunch(e.exec, h->st));
            h->hops_since_refresh = e.hsr_after;
            h->pending = true;
            return CG_OK;
        }
    cg_handle::GraphEntry e{};
    e.n_hops = n_hops;
    e.M = M;
    e.hsr_before = h->hops_since_refresh;
    CG_CUDA(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
    int rc = enqueue_run(h, n_hops, M, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->st, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        h->hops_since_refresh = e.hsr_before;
        return rc;
    }
    if (ce != cudaSuccess) return fail(CG_ECUDA, std::string("cudaStreamEndCapture: ") +
                                                     cudaGetErrorString(ce));
    e.hsr_after = h->hops_since_refresh;
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess)
        return fail(CG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    h->graphs.push_back(e);
    CG_CUDA(cudaGraphLaunch(e.exec, h->st));
    h->pending = true;
    return CG_OK;
}

int finish_run(cg_handle *h)
{
    // a group's counter blocks are contiguous: one copy per group (and one
    // per refresh error word) into pinned memory, queued behind the run
    for (size_t gi = 0; gi < h->groups.size(); ++gi) {
        const Group &g = h->groups[gi];
        CG_CUDA(cudaMemcpyAsync(h->h_ctr + g.first, h->reps[h->order[g.first]].d_ctr,
                                sizeof(DevCounters) * (size_t)g.count, cudaMemcpyDeviceToHost,
                                h->st));
        if (g.tc)
            CG_CUDA(cudaMemcpyAsync(h->h_err + gi, g.d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                    h->st));
    }
    CG_CUDA(cudaStreamSynchronize(h->st));
    h->pending = false;
    int rc = CG_OK;
    for (size_t k = 0; k < h->reps.size(); ++k) {
        const DevCounters &c = h->h_ctr[k];
        double e;
        std::memcpy(&e, &c.max_err_bits, 8);
        h->max_err_run = std::max(h->max_err_run, e);
        if (c.status == CG_ESTUCK) rc = fail(CG_ESTUCK, "a replica reached max rounds per hop");
        if (c.status == CG_ETIMEOUT)
            rc = fail(CG_ETIMEOUT, "a hop exceeded the device time limit");
    }
    for (size_t gi = 0; gi < h->groups.size(); ++gi) {
        const Group &g = h->groups[gi];
        if (g.tc && h->h_err[gi]) {
            CG_CUDA(cudaMemsetAsync(g.d_err, 0, sizeof(int), h->st));
            rc = fail(CG_ETIMEOUT, "a tensor-core refresh wait exceeded its time limit");
        }
    }
    return rc;
}

}  // namespace

namespace cg {
// Error message for entry points defined in other translation units.
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace cg

extern "C" {

const char *cg_version(void) { return "cg-pr 0.1 (sm_103a)"; }

const char *cg_last_error(void) { return g_err.c_str(); }

cg_handle *cg_create(int L, double nu, double W, double xi, int r_max, double T, double E,
                     uint64_t seed)
{
    cg_replica_desc d{};
    d.L = L; d.nu = nu; d.W = W; d.xi = xi; d.r_max = r_max; d.T = T; d.E = E;
    d.seed = seed; d.replica = 0;
    return create_impl(1, &d, nullptr, nullptr, 0);
}

cg_handle *cg_create_batch(int R, const cg_replica_desc *reps, const cg_opts *opts)
{
    return create_impl(R, reps, opts, nullptr, 0);
}

size_t cg_workspace_bytes(int R, const cg_replica_desc *reps, const cg_opts *opts)
{
    if (R <= 0 || !reps) return 0;
    // invalid descriptors (a random-site replica too large for a CTA among
    // them) give 0 before any geometry is built
    for (int k = 0; k < R; ++k)
        if (check_desc(reps[k]) != CG_OK) return 0;
    cg_opts o{};
    if (opts) o = *opts;
    return plan_bytes(R, reps, o);
}

cg_handle *cg_create_batch_ws(int R, const cg_replica_desc *reps, const cg_opts *opts,
                              void *workspace, size_t ws_bytes)
{
    if (!workspace) { fail(CG_EINVAL, "null workspace"); return nullptr; }
    return create_impl(R, reps, opts, workspace, ws_bytes);
}

void cg_destroy(cg_handle *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->st) cudaStreamSynchronize(h->st);
    for (void *p : h->allocs) cudaFree(p);
    if (h->d_log) cudaFree(h->d_log);
    if (h->d_trace) cudaFree(h->d_trace);
    for (auto &e : h->graphs) cudaGraphExecDestroy(e.exec);
    for (Group &g : h->groups) {
        if (g.st) cudaStreamDestroy(g.st);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    if (h->h_ctr) cudaFreeHost(h->h_ctr);
    if (h->h_err) cudaFreeHost(h->h_err);
    delete h;
}

int cg_num_replicas(const cg_handle *h) { return h ? (int)h->reps.size() : 0; }

int cg_site_positions(const cg_handle *h, int replica, double *x_host, double *y_host)
{
    const int rc = replica_index_ok(h, replica);
    if (rc) return rc;
    if (!x_host || !y_host) return fail(CG_EINVAL, "null output");
    const Rep &r = h->reps[replica];
    if (!r.random) return fail(CG_EINVAL, "a lattice replica's sites are its lattice points");
    std::memcpy(x_host, r.px.data(), sizeof(double) * (size_t)r.N);
    std::memcpy(y_host, r.py.data(), sizeof(double) * (size_t)r.N);
    return CG_OK;
}

int cg_num_sites(const cg_handle *h, int replica)
{
    if (!h || replica < 0 || replica >= (int)h->reps.size()) return 0;
    return h->reps[replica].N;
}

int cg_run_async(cg_handle *h, uint64_t n_hops, uint32_t M)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    return h->opts.use_graph ? enqueue_run_graph(h, n_hops, M) : enqueue_run(h, n_hops, M, false);
}

int cg_sync(cg_handle *h)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    return finish_run(h);
}

int cg_run(cg_handle *h, uint64_t n_hops, uint32_t M)
{
    int rc = cg_run_async(h, n_hops, M);
    if (rc) return rc;
    return finish_run(h);
}

int cg_run_logged(cg_handle *h, uint64_t n_hops, uint32_t M, cg_hop *log_host)
{
    if (!h || !log_host) return fail(CG_EINVAL, "null argument");
    const size_t R = h->reps.size();
    const size_t bytes = sizeof(cg_hop) * R * (size_t)n_hops;
    if (h->d_log) { cudaFree(h->d_log); h->d_log = nullptr; }
    if (bytes) CG_CUDA(cudaMalloc((void **)&h->d_log, bytes));
    // point every replica's log at its slice
    for (size_t k = 0; k < R; ++k) h->h_reps[k].log = h->d_log + k * n_hops;
    CG_CUDA(cudaMemcpyAsync(h->d_reps, h->h_reps.data(), sizeof(DevReplica) * R,
                            cudaMemcpyHostToDevice, h->st));
    int rc = enqueue_run(h, n_hops, M, true);
    int rc2 = rc ? rc : finish_run(h);
    for (size_t k = 0; k < R; ++k) h->h_reps[k].log = nullptr;
    CG_CUDA(cudaMemcpyAsync(h->d_reps, h->h_reps.data(), sizeof(DevReplica) * R,
                            cudaMemcpyHostToDevice, h->st));
    if (bytes) {
        CG_CUDA(cudaMemcpyAsync(log_host, h->d_log, bytes, cudaMemcpyDeviceToHost, h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
    }
    return rc2;
}

int cg_read_state(cg_handle *h, int replica, uint8_t *n_host, double *eps_host,
                  double *phi_host, cg_counters *c_host)
{
    int rc = replica_index_ok(h, replica);
    if (rc) return rc;
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    if (h->pending) CG_CUDA(cudaStreamSynchronize(h->st));
    const Rep &r = h->reps[replica];
    if (n_host) {
        std::vector<unsigned> w(r.words);
        CG_CUDA(cudaMemcpyAsync(w.data(), r.d_occ, 4 * w.size(), cudaMemcpyDeviceToHost, h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
        for (int s = 0; s < r.N; ++s) n_host[s] = (w[s >> 5] >> (s & 31)) & 1u;
    }
    if (eps_host && (rc = read_eps_host(h, r, eps_host))) return rc;
    if (phi_host) {
        CG_CUDA(cudaMemcpyAsync(phi_host, r.d_phi, 8 * (size_t)r.N, cudaMemcpyDeviceToHost, h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
    }
    if (c_host) {
        DevCounters dc;
        CG_CUDA(cudaMemcpyAsync(&dc, r.d_ctr, sizeof(dc), cudaMemcpyDeviceToHost, h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
        c_host->rounds = dc.rounds; c_host->hops = dc.hops; c_host->attempts = dc.attempts;
        c_host->evaluated = dc.evaluated; c_host->P = dc.P; c_host->energy = dc.energy;
        c_host->time = dc.time;
    }
    return CG_OK;
}

int cg_write_state(cg_handle *h, int replica, const uint8_t *n_host, const double *eps_host,
                   const double *phi_host, const cg_counters *c_host)
{
    int rc = replica_index_ok(h, replica);
    if (rc) return rc;
    if (!n_host) return fail(CG_EINVAL, "n_host is required");
    const Rep &r = h->reps[replica];
    long long cnt = 0;
    for (int s = 0; s < r.N; ++s) {
        if (n_host[s] > 1) return fail(CG_ESTATE, "occupations must be 0 or 1");
        cnt += n_host[s];
    }
    if (cnt != (long long)std::floor(r.d.nu * r.N + 0.5))
        return fail(CG_ESTATE, "occupation count differs from nu * N");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    if (h->pending) CG_CUDA(cudaStreamSynchronize(h->st));
    return load_state(h, replica, n_host, eps_host, phi_host, c_host);
}

int cg_group_replicas(const cg_handle *h, int group, int *replicas_out)
{
    if (!h || group < 0 || group >= (int)h->groups.size() || !replicas_out)
        return fail(CG_EINVAL, "bad group or null output");
    const Group &g = h->groups[group];
    for (int k = 0; k < g.count; ++k) replicas_out[k] = h->order[g.first + k];
    return g.count;
}

int cg_read_group_state(cg_handle *h, int group, uint32_t *occ_words_host, void *eps_host,
                        cg_counters *c_host)
{
    if (!h || group < 0 || group >= (int)h->groups.size()) return fail(CG_EINVAL, "bad group");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    if (h->pending) CG_CUDA(cudaStreamSynchronize(h->st));
    const Group &g = h->groups[group];
    const Rep &r0 = h->reps[h->order[g.first]];
    const size_t cnt = (size_t)g.count;
    const size_t rb = h->opts.precision == CG_FP64 ? 8 : 4;
    if (occ_words_host)
        CG_CUDA(cudaMemcpyAsync(occ_words_host, r0.d_occ, cnt * r0.words * 4,
                                cudaMemcpyDeviceToHost, h->st));
    if (eps_host)
        CG_CUDA(cudaMemcpyAsync(eps_host, r0.d_eps, cnt * r0.N * rb, cudaMemcpyDeviceToHost,
                                h->st));
    DevCounters *dc = h->h_ctr + g.first;      // pinned, group order
    if (c_host)
        CG_CUDA(cudaMemcpyAsync(dc, r0.d_ctr, cnt * sizeof(DevCounters), cudaMemcpyDeviceToHost,
                                h->st));
    CG_CUDA(cudaStreamSynchronize(h->st));
    for (size_t k = 0; c_host && k < cnt; ++k) {
        c_host[k].rounds = dc[k].rounds; c_host[k].hops = dc[k].hops;
        c_host[k].attempts = dc[k].attempts; c_host[k].evaluated = dc[k].evaluated;
        c_host[k].P = dc[k].P; c_host[k].energy = dc[k].energy;
        c_host[k].time = dc[k].time;
    }
    return CG_OK;
}

int cg_write_group_state(cg_handle *h, int group, const uint32_t *occ_words_host,
                         const void *eps_host, const cg_counters *c_host)
{
    if (!h || group < 0 || group >= (int)h->groups.size()) return fail(CG_EINVAL, "bad group");
    const Group &g = h->groups[group];
    const Rep &r0 = h->reps[h->order[g.first]];
    const size_t cnt = (size_t)g.count;
    const size_t rb = h->opts.precision == CG_FP64 ? 8 : 4;
    if (occ_words_host) {
        // every replica keeps nu N electrons and no bit beyond site N - 1
        for (size_t k = 0; k < cnt; ++k) {
            const Rep &r = h->reps[h->order[g.first + (int)k]];
            const uint32_t *w = occ_words_host + k * r0.words;
            long long n = 0;
            for (int q = 0; q < r0.words; ++q) n += __builtin_popcount(w[q]);
            if ((r0.N & 31) && (w[r0.words - 1] >> (r0.N & 31)))
                return fail(CG_ESTATE, "occupation bits beyond the last site");
            if (n != (long long)std::floor(r.d.nu * r.N + 0.5))
                return fail(CG_ESTATE, "occupation count differs from nu * N");
        }
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    if (h->pending) CG_CUDA(cudaStreamSynchronize(h->st));
    if (occ_words_host)
        CG_CUDA(cudaMemcpyAsync(r0.d_occ, occ_words_host, cnt * r0.words * 4,
                                cudaMemcpyHostToDevice, h->st));
    if (eps_host)
        CG_CUDA(cudaMemcpyAsync(r0.d_eps, eps_host, cnt * r0.N * rb, cudaMemcpyHostToDevice,
                                h->st));
    if (c_host) {
        // the public counters are replaced; the library's own fields (chunk
        // statistics, refresh record, trace state, phase clocks) are kept
        DevCounters *dc = h->h_ctr + g.first;  // pinned, group order
        CG_CUDA(cudaMemcpyAsync(dc, r0.d_ctr, cnt * sizeof(DevCounters),
                                cudaMemcpyDeviceToHost, h->st));
        CG_CUDA(cudaStreamSynchronize(h->st));
        for (size_t k = 0; k < cnt; ++k) {
            dc[k].rounds = c_host[k].rounds; dc[k].hops = c_host[k].hops;
            dc[k].attempts = c_host[k].attempts; dc[k].evaluated = c_host[k].evaluated;
            dc[k].P = c_host[k].P; dc[k].energy = c_host[k].energy;
            dc[k].time = c_host[k].time;
        }
        CG_CUDA(cudaMemcpyAsync(r0.d_ctr, dc, cnt * sizeof(DevCounters),
                                cudaMemcpyHostToDevice, h->st));
    }
    CG_CUDA(cudaStreamSynchronize(h->st));
    return CG_OK;
}

int cg_observables(cg_handle *h, int replica, cg_obs *out)
{
    int rc = replica_index_ok(h, replica);
    if (rc) return rc;
    if (!out) return fail(CG_EINVAL, "null output");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    if (h->pending) CG_CUDA(cudaStreamSynchronize(h->st));
    const Rep &r = h->reps[replica];
    DevCounters dc;
    CG_CUDA(cudaMemcpyAsync(&dc, r.d_ctr, sizeof(dc), cudaMemcpyDeviceToHost, h->st));
    CG_CUDA(cudaStreamSynchronize(h->st));
    std::memset(out, 0, sizeof(*out));
    out->c.rounds = dc.rounds; out->c.hops = dc.hops; out->c.attempts = dc.attempts;
    out->c.evaluated = dc.evaluated; out->c.P = dc.P; out->c.energy = dc.energy;
    out->c.time = dc.time;
    out->Gamma = gamma_of(r, h->opts);
    out->time = h->opts.time_mode == CG_TIME_GAUSSIAN ? dc.time
                                                      : (double)dc.attempts / out->Gamma;
    out->acceptance = dc.attempts ? (double)dc.hops / (double)dc.attempts : 0.0;
    out->energy_per_site = dc.energy / (double)r.N;
    std::memcpy(&out->max_eps_err_last_refresh, &dc.max_err_bits, 8);
    out->refreshes = dc.refreshes;
    out->cycles_reject = dc.cycles_reject;
    out->cycles_update = dc.cycles_update;
    return CG_OK;
}

int cg_refresh(cg_handle *h)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    int rc = refresh_all(h);
    if (rc) return rc;
    CG_CUDA(cudaStreamSynchronize(h->st));
    return CG_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: per lattice-size group, time the persistent launch for each
// cluster size (CTAs per replica), CTA size and M on a copy of the state, keep
// the fastest.  Results are cached in the JSON file named by $CG_TUNE_CACHE
// (flat map key -> {"threads", "M", "cluster"}).
// ---------------------------------------------------------------------------

static std::string tune_key(const cg_handle *h, const Group &g)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, h->device);
    const Rep &r = h->reps[h->order[g.first]];
    char buf[512];
    // a forced cluster size is part of the key; otherwise the tuner picks it
    char cl[16];
    if (h->opts.cluster_size > 1)
        std::snprintf(cl, sizeof(cl), "%d", h->opts.cluster_size);
    else
        std::snprintf(cl, sizeof(cl), "auto");
    std::snprintf(buf, sizeof(buf), "%s|L=%d|dim=%d|prec=%s|cluster=%s|rmax=%d|T=%.6g|R=%d|pair=%.6g",
                  prop.name, g.L, g.dim, h->opts.precision == CG_FP64 ? "fp64" : "fp32", cl,
                  r.d.r_max, r.d.T, g.count, h->opts.pair_frac);
    return std::string(buf);
}

static bool tune_cache_lookup(const std::string &text, const std::string &key, int *threads,
                              unsigned *M, int *cluster)
{
    const std::string pat = "\"" + key + "\": {\"threads\": ";
    const size_t p = text.find(pat);
    if (p == std::string::npos) return false;
    int t = 0, c = 0;
    unsigned m = 0;
    if (std::sscanf(text.c_str() + p + pat.size(), "%d, \"M\": %u, \"cluster\": %d", &t, &m,
                    &c) != 3)
        return false;
    *threads = t;
    *M = m;
    *cluster = c;
    return true;
}

// Cluster sizes a group can run with (CTAs per replica): the size chosen at
// creation when the caller forced one; else 1 (when eps fits one CTA) and
// every 2, 4, 8 whose per-CTA shared memory fits (on lattices: that divides
// L as the row split needs), each with that shared-memory size.
static std::vector<std::pair<int, int>> cluster_candidates(const cg_handle *h, const Group &g)
{
    std::vector<std::pair<int, int>> out;
    if (h->opts.cluster_size > 1) {
        out.push_back({g.cluster, g.smem});
        return out;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    const int budget = optin - (h->opts.pair_frac > 0.0 ? 3072 : 2048);
    for (int c = 1; c <= 8; c *= 2) {
        if (c > 1 && !g.random && (g.L % (g.dim == 3 ? c : 2 * c) != 0 || g.L < 16)) continue;
        int sm = 0;
        for (int k = 0; k < g.count; ++k)
            sm = std::max(sm, persistent_smem(h->reps[h->order[g.first + k]], h->opts.precision, c));
        if (sm <= budget) out.push_back({c, sm});
    }
    return out;
}

int cg_autotune(cg_handle *h, uint32_t hops_per_trial)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (hops_per_trial == 0) hops_per_trial = 256;
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    CG_CUDA(cudaStreamSynchronize(h->st));
    const char *path = std::getenv("CG_TUNE_CACHE");
    std::string cache;
    if (path) {
        if (FILE *f = std::fopen(path, "r")) {
            char buf[4096];
            size_t n;
            while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) cache.append(buf, n);
            std::fclose(f);
        }
    }
    const int rb = h->opts.precision == CG_FP64 ? 8 : 4;
    struct Shape { int threads; unsigned M; int cluster; };
    std::vector<std::pair<std::string, Shape>> found;
    cudaEvent_t e0, e1;
    CG_CUDA(cudaEventCreate(&e0));
    CG_CUDA(cudaEventCreate(&e1));
    int rc = CG_OK;
    for (Group &g : h->groups) {
        const std::string key = tune_key(h, g);
        const std::vector<std::pair<int, int>> cands = cluster_candidates(h, g);
        int ct = 0, cc = 0;
        unsigned cM = 0;
        if (tune_cache_lookup(cache, key, &ct, &cM, &cc)) {
            for (const auto &c : cands)
                if (c.first == cc) {
                    g.cluster = cc;
                    g.smem = c.second;
                    g.threads = ct;
                    g.M = cM;
                    g.tuned = true;
                }
            if (g.tuned) continue;
        }
        // snapshot of the group's state (eps, bitmask, counters per replica)
        const Rep &r0 = h->reps[h->order[g.first]];
        const size_t per = (size_t)r0.N * rb + (size_t)r0.words * 4 + sizeof(DevCounters);
        char *snap = nullptr;
        if (cudaMalloc((void **)&snap, per * g.count) != cudaSuccess) {
            rc = fail(CG_ENOMEM, "autotune snapshot allocation failed");
            break;
        }
        auto copy_group = [&](bool save) -> cudaError_t {
            for (int k = 0; k < g.count; ++k) {
                const Rep &r = h->reps[h->order[g.first + k]];
                char *s = snap + per * k;
                const size_t be = (size_t)r.N * rb, bo = (size_t)r.words * 4;
                cudaError_t e;
                if ((e = cudaMemcpyAsync(save ? s : r.d_eps, save ? r.d_eps : s, be,
                                         cudaMemcpyDeviceToDevice, h->st)))
                    return e;
                if ((e = cudaMemcpyAsync(save ? s + be : (void *)r.d_occ,
                                         save ? (void *)r.d_occ : s + be, bo,
                                         cudaMemcpyDeviceToDevice, h->st)))
                    return e;
                if ((e = cudaMemcpyAsync(save ? s + be + bo : (void *)r.d_ctr,
                                         save ? (void *)r.d_ctr : s + be + bo,
                                         sizeof(DevCounters), cudaMemcpyDeviceToDevice, h->st)))
                    return e;
            }
            return cudaStreamSynchronize(h->st);
        };
        cudaError_t ce = copy_group(true);
        double best = -1.0;
        int best_t = g.threads, best_c = g.cluster, best_smem = g.smem;
        unsigned best_M = g.M;
        const int shapes[4] = {256, 384, 512, 1024};
        const unsigned Ms[4] = {1024, 4096, 16384, 65536};
        std::vector<DevCounters> cs(g.count);
        for (const auto &cand : cands) {
            const int c = cand.first;
            for (int ti = 0; ti < 4 && ce == cudaSuccess; ++ti) {
                const int t = shapes[ti];
                // the single-CTA update needs L/2 base columns (L on the cubic
                // lattice); the cluster kernel maps a thread to a column and
                // is built for 512 and 1024 threads; the random-site kernels
                // take any L, the cluster form 256, 512 or 1024 threads
                if (g.random) {
                    if (c > 1 && t == 384) continue;
                } else {
                    if (t < g.L / 2 || (g.dim == 3 && t < g.L)) continue;
                    if (c > 1 && (t < 512 || t < g.L)) continue;
                }
                for (int mi = 0; mi < 4 && ce == cudaSuccess; ++mi) {
                    Group trial = g;
                    trial.threads = t;
                    trial.cluster = c;
                    trial.smem = cand.second;
                    cudaEventRecord(e0, h->st);
                    int lrc = launch_group(h, trial, hops_per_trial, Ms[mi], 0, h->st);
                    cudaEventRecord(e1, h->st);
                    ce = cudaStreamSynchronize(h->st);
                    if (lrc || ce != cudaSuccess) break;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    // a trial counts only when every replica of the group
                    // completed its hops (none stuck or past its time limit)
                    bool ok = ms > 0.f;
                    for (int k = 0; k < g.count && ok; ++k) {
                        const Rep &r = h->reps[h->order[g.first + k]];
                        ce = cudaMemcpy(&cs[k], r.d_ctr, sizeof(DevCounters),
                                        cudaMemcpyDeviceToHost);
                        ok = ce == cudaSuccess && cs[k].status == CG_OK;
                    }
                    if (ce != cudaSuccess) break;
                    const double rate = ok ? (double)g.count * hops_per_trial / (ms * 1e-3) : 0.0;
                    if (rate > best) {
                        best = rate;
                        best_t = t;
                        best_M = Ms[mi];
                        best_c = c;
                        best_smem = cand.second;
                    }
                    ce = copy_group(false);   // restore: tuning leaves the chains untouched
                }
            }
        }
        cudaFree(snap);
        if (ce != cudaSuccess) {
            rc = fail(CG_ECUDA, std::string("autotune: ") + cudaGetErrorString(ce));
            break;
        }
        g.threads = best_t;
        g.M = best_M;
        g.cluster = best_c;
        g.smem = best_smem;
        g.tuned = true;
        found.push_back({key, {best_t, best_M, best_c}});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto &e : h->graphs) cudaGraphExecDestroy(e.exec);   // shapes changed
    h->graphs.clear();
    if (rc == CG_OK && path && !found.empty()) {
        // rewrite the cache with the old entries plus the new ones
        std::string body;
        size_t p = cache.find('{');
        size_t q = cache.rfind('}');
        if (p != std::string::npos && q != std::string::npos && q > p) {
            body = cache.substr(p + 1, q - p - 1);
            while (!body.empty() && (body.back() == '\n' || body.back() == ' ')) body.pop_back();
        }
        if (FILE *f = std::fopen(path, "w")) {
            std::fprintf(f, "{");
            bool first = body.find('"') == std::string::npos;
            if (!first) std::fprintf(f, "%s", body.c_str());
            for (auto &e : found) {
                std::fprintf(f, "%s\n  \"%s\": {\"threads\": %d, \"M\": %u, \"cluster\": %d}",
                             first ? "" : ",", e.first.c_str(), e.second.threads, e.second.M,
                             e.second.cluster);
                first = false;
            }
            std::fprintf(f, "\n}\n");
            std::fclose(f);
        }
    }
    return rc;
}

int cg_set_trace(cg_handle *h, double first_time, double points_per_decade, int capacity)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (!(first_time > 0.0) || !(points_per_decade > 0.0) || capacity < 1)
        return fail(CG_EINVAL, "need first_time > 0, points_per_decade > 0, capacity >= 1");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    CG_CUDA(cudaStreamSynchronize(h->st));
    const size_t R = h->reps.size();
    if (h->d_trace) {
        cudaFree(h->d_trace);
        h->d_trace = nullptr;
    }
    CG_CUDA(cudaMalloc((void **)&h->d_trace, sizeof(cg_trace_point) * R * (size_t)capacity));
    const double ratio = std::pow(10.0, 1.0 / points_per_decade);
    for (size_t k = 0; k < R; ++k) {
        const Rep &r = h->reps[k];
        DevCounters c;
        CG_CUDA(cudaMemcpy(&c, r.d_ctr, sizeof(c), cudaMemcpyDeviceToHost));
        // the first point is the present state; later points at first_time * ratio^n
        cg_trace_point p0{c.attempts, c.hops, c.P, c.energy};
        CG_CUDA(cudaMemcpy(h->d_trace + k * capacity, &p0, sizeof(p0), cudaMemcpyHostToDevice));
        const double Gamma = gamma_of(r, h->opts);
        c.trace_count = 1;
        c.trace_cap = capacity;
        c.trace_ratio = ratio;
        c.trace_next = std::max((double)c.attempts + 1.0, first_time * Gamma);
        CG_CUDA(cudaMemcpy(r.d_ctr, &c, sizeof(c), cudaMemcpyHostToDevice));
        h->h_reps[k].trace = h->d_trace + k * capacity;
    }
    CG_CUDA(cudaMemcpy(h->d_reps, h->h_reps.data(), sizeof(DevReplica) * R,
                       cudaMemcpyHostToDevice));
    for (auto &e : h->graphs) cudaGraphExecDestroy(e.exec);   // descriptors changed
    h->graphs.clear();
    h->trace_cap = capacity;
    return CG_OK;
}

int cg_read_trace(cg_handle *h, int replica, cg_trace_point *out_host, int cap)
{
    int rc = replica_index_ok(h, replica);
    if (rc) return rc;
    if (!out_host || cap < 0) return fail(CG_EINVAL, "bad output buffer");
    if (!h->d_trace) return 0;
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    CG_CUDA(cudaStreamSynchronize(h->st));
    DevCounters c;
    CG_CUDA(cudaMemcpy(&c, h->reps[replica].d_ctr, sizeof(c), cudaMemcpyDeviceToHost));
    const int n = std::min(cap, c.trace_count);
    if (n > 0)
        CG_CUDA(cudaMemcpy(out_host, h->d_trace + (size_t)replica * h->trace_cap,
                           sizeof(cg_trace_point) * n, cudaMemcpyDeviceToHost));
    return n;
}

int cg_num_groups(const cg_handle *h) { return h ? (int)h->groups.size() : 0; }

int cg_group_shape(const cg_handle *h, int index, int *L, int *threads, unsigned *M,
                   int *cluster)
{
    if (!h || index < 0 || index >= (int)h->groups.size())
        return fail(CG_EINVAL, "group index out of range");
    const Group &g = h->groups[index];
    if (L) *L = g.L;
    if (threads) *threads = g.threads;
    if (M) *M = g.M;
    if (cluster) *cluster = g.cluster;
    return CG_OK;
}

int cg_refresh_async(cg_handle *h)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    int rc = refresh_all(h);
    if (rc) return rc;
    h->pending = true;
    return CG_OK;
}

int cg_microbench(int kind, int device, double *result)
{
    if (!result || kind < 0 || kind > 7) return fail(CG_EINVAL, "bad microbenchmark kind");
    int rc = microbench(kind, device, result);
    if (rc) return fail(rc, "microbenchmark failed");
    return CG_OK;
}

int cg_set_toy_acceptance(cg_handle *h, double A0)
{
    if (!h) return fail(CG_EINVAL, "null handle");
    if (A0 < 0) { h->toy = 0; h->toy_A0 = 0; return CG_OK; }
    if (!(A0 <= 1.0)) return fail(CG_EINVAL, "A0 must be in [0, 1]");
    for (const Rep &r : h->reps)
        if (r.random) return fail(CG_EINVAL, "random sites have no constant-acceptance mode");
    h->toy = 1;
    h->toy_A0 = A0;
    return CG_OK;
}

int cg_debug_philox(const uint32_t *ctr_host, const uint32_t *key_host, uint32_t *out_host,
                    int n)
{
    if (n <= 0 || !ctr_host || !key_host || !out_host) return fail(CG_EINVAL, "bad arguments");
    uint32_t *d = nullptr;
    CG_CUDA(cudaMalloc((void **)&d, sizeof(uint32_t) * 10 * (size_t)n));
    uint32_t *dc = d, *dk = d + 4 * (size_t)n, *dout = d + 6 * (size_t)n;
    cudaMemcpy(dc, ctr_host, 16 * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, key_host, 8 * (size_t)n, cudaMemcpyHostToDevice);
    cudaError_t e = launch_debug_philox(dc, dk, dout, n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out_host, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CG_ECUDA, cudaGetErrorString(e));
    return CG_OK;
}

int cg_debug_exp(const double *x_host, double *out_host, int n)
{
    if (n <= 0 || !x_host || !out_host) return fail(CG_EINVAL, "bad arguments");
    double *d = nullptr;
    CG_CUDA(cudaMalloc((void **)&d, 16 * (size_t)n));
    cudaMemcpy(d, x_host, 8 * (size_t)n, cudaMemcpyHostToDevice);
    cudaError_t e = launch_debug_exp(d, d + n, n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out_host, d + n, 8 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CG_ECUDA, cudaGetErrorString(e));
    return CG_OK;
}

int cg_debug_gauss(const uint64_t *seed_host, const uint32_t *replica_host,
                   const uint64_t *hops_host, double *z_host, int n)
{
    if (n <= 0 || !seed_host || !replica_host || !hops_host || !z_host)
        return fail(CG_EINVAL, "bad arguments");
    char *d = nullptr;
    CG_CUDA(cudaMalloc((void **)&d, 28 * (size_t)n));
    uint64_t *ds = (uint64_t *)d, *dh = (uint64_t *)(d + 8 * (size_t)n);
    double *dz = (double *)(d + 16 * (size_t)n);
    uint32_t *dr = (uint32_t *)(d + 24 * (size_t)n);
    cudaError_t e = cudaMemcpy(ds, seed_host, 8 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dh, hops_host, 8 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dr, replica_host, 4 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_gauss(ds, dr, dh, dz, n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(z_host, dz, 8 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CG_ECUDA, cudaGetErrorString(e));
    return CG_OK;
}

int cg_eps_histogram(cg_handle *h, int first, int count, int nbins, double lo, double hi,
                     uint64_t *counts_dev)
{
    if (!h || !counts_dev) return fail(CG_EINVAL, "cg_eps_histogram: null handle or output");
    if (first < 0 || count < 1 || first + count > (int)h->reps.size())
        return fail(CG_EINVAL, "cg_eps_histogram: replicas out of range");
    if (nbins < 1 || nbins > 4096) return fail(CG_EINVAL, "cg_eps_histogram: nbins must be 1..4096");
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi))
        return fail(CG_EINVAL, "cg_eps_histogram: need finite lo < hi");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    int max_N = 0;
    for (int k = first; k < first + count; ++k) max_N = std::max(max_N, h->reps[k].N);
    const double scale = (double)nbins / (hi - lo);
    CG_CUDA(launch_eps_histogram(h->d_reps + first, count, max_N, h->opts.precision, nbins, lo,
                                 scale, reinterpret_cast<unsigned long long *>(counts_dev), h->st));
    return CG_OK;
}

int cg_debug_tower(cg_handle *h, int replica, const uint32_t *x1_host, int32_t *v_host, int n)
{
    if (!h || n <= 0 || !x1_host || !v_host) return fail(CG_EINVAL, "bad arguments");
    if (replica < 0 || replica >= (int)h->reps.size()) return fail(CG_EINVAL, "replica out of range");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(CG_ECUDA, "cudaSetDevice failed");
    if (h->reps[replica].random)
        return fail(CG_EINVAL, "a random-site replica draws from its partner lists");
    const Tables &t = *h->reps[replica].tab;
    char *d = nullptr;
    CG_CUDA(cudaMalloc((void **)&d, 8 * (size_t)n));
    uint32_t *dx = (uint32_t *)d;
    int *dv = (int *)(d + 4 * (size_t)n);
    cudaError_t e = cudaMemcpy(dx, x1_host, 4 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_tower(t.d_guide, t.d_thr, t.V, dx, dv, n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(v_host, dv, 4 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CG_ECUDA, cudaGetErrorString(e));
    return CG_OK;
}

}  // extern "C"
