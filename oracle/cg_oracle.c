/*
 * cg_oracle.c -- plain, slow, serial CPU oracle of the mixed rejection KMC
 * chain for the lattice Coulomb glass (Ferrero, Kolton & Palassini,
 * "Parallel kinetic Monte Carlo simulation of Coulomb glasses").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code with the CUDA library; both follow the same
 * written definition (the paper plus the readings listed below).
 *
 * Every floating-point quantity is IEEE binary64.  Compile with
 * -ffp-contract=off (no fused multiply-add) and without -ffast-math, so that
 * each + - * / sqrt is one correctly rounded operation in source order.
 *
 * What each function follows:
 *   orc_philox        Philox-4x32-10 of Salmon, Moraes, Dror & Shaw (SC'11,
 *                     "Parallel random numbers: as easy as 1, 2, 3"); the
 *                     paper draws its random numbers from Philox (section
 *                     "Hopping conduction in the Coulomb glass", GPU
 *                     implementation paragraph).
 *   orc_cg_exp        exp(x) by Cody & Waite's additive range reduction
 *                     (Software Manual for the Elementary Functions, 1980)
 *                     followed by the Taylor series to degree 13.
 *   orc_new           Eq. 1 (Hamiltonian, filling, disorder), the tunnelling
 *                     factor of Eq. 2 and the rate normalisation Gamma, the
 *                     lattice model with toroidal boundaries and minimum image
 *                     (section "Results for the lattice model in two
 *                     dimensions").
 *   orc_eps_scratch   the single-particle energies below Eq. 2:
 *                     eps_i = phi_i + sum_j (n_j - nu) / r_ij.
 *   orc_eval_label    steps 1-2 of the mixed PR algorithm (proposal by the
 *                     tunnelling factor, acceptance by the activation factor
 *                     Gamma^A = theta * min[1, exp(-dH/T)]) for one label.
 *   orc_run           the serial rejection algorithm (section "Parallel
 *                     rejection algorithm", steps 1-2) driven label by label;
 *                     on the first accepting label it executes step 3 of the
 *                     mixed PR algorithm (3a commit, 3b dipole and local-energy
 *                     update, 3c time through the attempt count).
 *
 * Readings of the paper taken here:
 *   R1  Philox key = (seed lo 32, seed hi 32); proposal counter for round r,
 *       label k (0-based) of replica c = (k, r lo 32, r hi 32, c); three of
 *       the four output words are used (site, displacement, acceptance).
 *   R2  Displacements: all (dx,dy) with 0 < dx^2+dy^2 <= r_max^2 (r_max
 *       strictly below L/2), ordered dy outer ascending, dx inner ascending;
 *       on the cubic lattice all (dx,dy,dz) with 0 < dx^2+dy^2+dz^2 <=
 *       r_max^2, dz outermost (the plane dz = 0 is the square lattice's).
 *       Tower sampling over integer weights W_k = floor(2^32 w_k / Z),
 *       w_k = exp(-2 r_k / xi), Z = sum_k w_k; the sampled vector is the
 *       smallest k with x1 < C_k (C_k the running sum); x1 >= C_{V-1} is a
 *       null proposal (rejected, counted as an attempt).
 *   R3  The attempt count advances by (p-1) M + q per executed hop (q 1-based):
 *       the paper's "m = pM + q" (step 3c) disagrees with its Fig. 1 example
 *       and with <m> = 1/A; every round without an accept adds M.
 *   R4  Time is the deterministic t = attempts / Gamma with Gamma = N * Z,
 *       the rule the paper used for its figures (Fig. 3 caption).
 *   R5  Disorder phi_s = W (u - 1/2), u = (x0 + 1/2) 2^-32 from counter
 *       (s, 1, 0xFFFFFFFF, c): W is the full width of the interval.
 *   R6  Initial occupation: sites sorted by (x0 of counter (s, 2, 0xFFFFFFFF,
 *       c), s) ascending; the first nu*N sites are occupied.
 *   R7  Accept iff dH <= 0 or u < exp(-dH/T), u = (x2 + 1/2) 2^-32, with the
 *       exp of orc_cg_exp; exp(x) for x < -23 is taken as 0 (it is below the
 *       smallest u, so the decision is unchanged).
 *   R8  The 1/r table holds 0 at zero displacement, which makes the three
 *       cases of step 3b one formula: eps_l += 1/r_lj - 1/r_li.
 *   R9  dH = ((eps_j - eps_i) - 1/r_ij) - E * dx evaluated in that order.
 *   R10 Incremental energy: E_tot += dH of each executed hop; the dipole P
 *       accumulates the hop's minimum-image dx (unwrapped).
 *   R13 Stochastic time (step 3c, optional; R4 stays the default): each
 *       executed hop adds dt = max(0, (m + sqrt(m) z) / Gamma), m = (p-1)M + q,
 *       z standard normal by Box-Muller from the Philox block of counter
 *       (h lo, h hi, 0xFFFFFFFE, c), h the number of hops executed before
 *       this one: z = sqrt(-2 ln u1) cos(2 pi u2), u1 = (x0 + 1/2) 2^-32,
 *       u2 = x1 2^-32.  The paper's Gaussian can go negative for small m and
 *       it is silent on that case; it is clamped at zero.
 *   R15 Two-electron hops (the multi-electron hops the paper names as an
 *       extension, optional; square lattice).  A label is a pair proposal
 *       iff its fourth Philox word x3 < T_p = floor(p2 2^32).  A second
 *       Philox block of counter (k, r lo, r hi | 2^31, c) gives y0 -> ex,
 *       y2 -> ey (and y3 -> ez on the cubic lattice), each
 *       floor(y (2R+1) / 2^32) - R (an offset e uniform on the square
 *       [-R, R]^2 or the cube [-R, R]^3), and y1 -> a second tower vector d2.  The
 *       second electron moves k = i + e -> l = k + d2.  The pair passes
 *       theta iff n_i = n_k = 1, n_j = n_l = 0, 0 < |e|^2 <= R^2 and
 *       0 < |e'|^2 <= R^2 with e' = e + d2 - d1 (the reverse move's offset),
 *       so every pair proposal and its reverse have the same probability.
 *       dH = (dH1 + dH2) + ((1/r_lj - 1/r_li) - (1/r_kj - 1/r_ki)),
 *       dH1 = ((eps_j - eps_i) - 1/r_ij) - E dx1, dH2 likewise for k -> l:
 *       the exact change of Eq. 1.  The commit applies the two single-hop
 *       eps updates in turn; P gains dx1 + dx2; Gamma = N Z / (1 - T_p 2^-32).
 *   R16 Random sites (the random-site Coulomb glass, optional): N = L^2 sites
 *       at x = L (x0 + 1/2) 2^-32, y = L (x1 + 1/2) 2^-32 from the Philox
 *       block of counter (s, 3, 0xFFFFFFFF, c) in the L x L periodic box;
 *       1/r with the minimum-image displacement (dx = x_t - x_s, shifted by
 *       -L or +L when beyond L/2).  The hop partners of i are the j != i with
 *       r_ij <= r_max in ascending j, weights w = exp(-2 r / xi), Z_i their sum,
 *       Zmax = max_i Z_i and integer weights floor(2^32 w / Zmax): a label
 *       draws i = floor(x0 N / 2^32) and the smallest partner k with
 *       x1 < C_k (C the running sums over i's list; none: a null proposal).
 *       The proposal probability W_ij 2^-32 / N is symmetric exactly, and
 *       Gamma = N Zmax.  dH = ((eps_j - eps_i) - 1/r_ij) - E dx_ij with the
 *       real minimum-image dx_ij; the dipole is not accumulated.
 *
 * Geometry is a general Lx x Ly x Lz torus (Ly = Lz = 1 gives a ring, Lz = 1
 * the square lattice, Lx = Ly = Lz the cubic lattice of the 3D extension) so
 * that tiny
 * systems can be enumerated exactly; the library itself builds L x L and
 * L x L x L.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ESTUCK -5

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10                                                            */
/* ------------------------------------------------------------------------ */

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t prod0, prod1;
        uint32_t n0, n1, n2, n3;
        if (round > 0) {            /* key schedule: Weyl increments */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        n1 = (uint32_t)prod1;
        n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* exp by Cody-Waite reduction + Taylor series                               */
/* ------------------------------------------------------------------------ */

/* ln 2 = 0.693147180559945309417232121458176568...; LN2_HI keeps its leading
 * 29 significant bits, so k * LN2_HI is exact for |k| < 2^24, and LN2_LO is
 * the rest, rounded to double. */
static const double ORC_LN2_HI = 0x1.62e42ffp-1;
static const double ORC_LN2_LO = -0x1.718432a1b0e26p-35;
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;

/* exp(x) for -745 < x <= 0 (the only range this model needs). */
double orc_exp_core(double x)
{
    double kd, r, p;
    int n;
    kd = nearbyint(x * ORC_INV_LN2);
    r = (x - kd * ORC_LN2_HI) - kd * ORC_LN2_LO;
    /* Horner form of sum_{n=0}^{13} r^n / n!, coefficients 1/n! rounded */
    p = 1.0 / 6227020800.0;              /* 1/13! */
    {
        static const double fact[13] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0,
                                        5040.0, 40320.0, 362880.0, 3628800.0,
                                        39916800.0, 479001600.0};
        for (n = 12; n >= 0; --n) {
            double t = p * r;
            p = t + 1.0 / fact[n];
        }
    }
    return ldexp(p, (int)kd);
}

/* The acceptance exponential (reading R7). */
double orc_cg_exp(double x)
{
    if (x < -23.0) return 0.0;
    return orc_exp_core(x);
}

/* ---- stochastic time increment (reading R13) ---- */

/* Natural logarithm of a normal x > 0: x = 2^k m with m in [sqrt(1/2),
 * sqrt(2)); ln m = 2 atanh(f), f = (m - 1)/(m + 1) (|f| <= 0.1716), by the
 * odd series f + f^3/3 + ... + f^23/23 (the next term is below 3e-21);
 * ln x = k LN2_HI + (k LN2_LO + ln m).  The coefficients 1/(2n+1) are
 * rounded to binary64. */
double orc_log(double x)
{
    uint64_t b;
    int k;
    double m, f, s, p, lm;
    memcpy(&b, &x, 8);
    k = (int)((b >> 52) & 0x7ff) - 1023;
    b = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;   /* m in [1, 2) */
    memcpy(&m, &b, 8);
    if (m > 0x1.6a09e667f3bcdp+0) {                            /* sqrt(2) */
        m = m * 0.5;
        k += 1;
    }
    f = (m - 1.0) / (m + 1.0);
    s = f * f;
    p = 0x1.642c8590b2164p-5;               /* 1/23 */
    p = p * s + 0x1.8618618618618p-5;       /* 1/21 */
    p = p * s + 0x1.af286bca1af28p-5;       /* 1/19 */
    p = p * s + 0x1.e1e1e1e1e1e1ep-5;       /* 1/17 */
    p = p * s + 0x1.1111111111111p-4;       /* 1/15 */
    p = p * s + 0x1.3b13b13b13b14p-4;       /* 1/13 */
    p = p * s + 0x1.745d1745d1746p-4;       /* 1/11 */
    p = p * s + 0x1.c71c71c71c71cp-4;       /* 1/9 */
    p = p * s + 0x1.2492492492492p-3;       /* 1/7 */
    p = p * s + 0x1.999999999999ap-3;       /* 1/5 */
    p = p * s + 0x1.5555555555555p-2;       /* 1/3 */
    p = p * s + 1.0;
    lm = (2.0 * f) * p;
    return (double)k * ORC_LN2_HI + ((double)k * ORC_LN2_LO + lm);
}

/* cos(2 pi u) for u in [0, 1): v = u - rint(u), q = rint(4 v) and
 * w = v - q/4 in [-1/8, 1/8] are exact; theta = 2 pi w; cos(2 pi u) is
 * cos(theta), -sin(theta), -cos(theta) or sin(theta) for q = 0, 1, 2, 3
 * (mod 4), from the Taylor series of cos to theta^16 and of sin to theta^17
 * on |theta| <= pi/4 (remainders below 3e-18). */
double orc_cos2pi(double u)
{
    double v = u - rint(u);
    double q = rint(4.0 * v);
    double w = v - 0.25 * q;
    double t = 0x1.921fb54442d18p+2 * w;    /* 2 pi */
    double s = t * t, p, r;
    int qi = ((int)q) & 3;
    if (qi == 0 || qi == 2) {
        p = 0x1.ae7f3e733b81fp-45;              /*  1/16! */
        p = p * s + -0x1.93974a8c07c9dp-37;     /* -1/14! */
        p = p * s + 0x1.1eed8eff8d898p-29;      /*  1/12! */
        p = p * s + -0x1.27e4fb7789f5cp-22;     /* -1/10! */
        p = p * s + 0x1.a01a01a01a01ap-16;      /*  1/8! */
        p = p * s + -0x1.6c16c16c16c17p-10;     /* -1/6! */
        p = p * s + 0x1.5555555555555p-5;       /*  1/4! */
        p = p * s + -0x1.0p-1;                  /* -1/2! */
        p = p * s + 1.0;
        r = p;
    } else {
        p = 0x1.952c77030ad4ap-49;              /*  1/17! */
        p = p * s + -0x1.ae7f3e733b81fp-41;     /* -1/15! */
        p = p * s + 0x1.6124613a86d09p-33;      /*  1/13! */
        p = p * s + -0x1.ae64567f544e4p-26;     /* -1/11! */
        p = p * s + 0x1.71de3a556c734p-19;      /*  1/9! */
        p = p * s + -0x1.a01a01a01a01ap-13;     /* -1/7! */
        p = p * s + 0x1.1111111111111p-7;       /*  1/5! */
        p = p * s + -0x1.5555555555555p-3;      /* -1/3! */
        p = p * s + 1.0;
        r = t * p;
    }
    return (qi == 1 || qi == 2) ? -r : r;
}

/* Standard normal deviate of executed hop h of a replica (Box-Muller on the
 * Philox block of counter (h lo, h hi, 0xFFFFFFFE, replica)). */
double orc_gauss(uint64_t seed, uint32_t replica, uint64_t h)
{
    uint32_t ctr[4], key[2], x[4];
    double u1, u2;
    ctr[0] = (uint32_t)h;
    ctr[1] = (uint32_t)(h >> 32);
    ctr[2] = 0xFFFFFFFEu;
    ctr[3] = replica;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    orc_philox(ctr, key, x);
    u1 = ((double)x[0] + 0.5) * 0x1p-32;
    u2 = (double)x[1] * 0x1p-32;
    return sqrt(-2.0 * orc_log(u1)) * orc_cos2pi(u2);
}

/* Time increment of one executed hop that took m attempts (reading R13). */
double orc_time_increment(double Gamma, uint64_t m, double z)
{
    double dm = (double)m;
    double d = dm + sqrt(dm) * z;
    if (d < 0.0) d = 0.0;
    return d / Gamma;
}

/* ------------------------------------------------------------------------ */
/* Chain state                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t rounds;      /* global round counter r of this replica */
    uint64_t hops;        /* executed hops */
    uint64_t attempts;    /* serial-equivalent attempts */
    uint64_t evaluated;   /* labels evaluated (== attempts for the serial chain) */
    int64_t P;            /* dipole moment, unwrapped (sum of hop dx) */
    double energy;        /* H_0 + sum of executed dH */
    double time;          /* stochastic time (reading R13); 0 in the default mode */
} orc_counters;

typedef struct {
    uint32_t i, j;        /* origin and destination site */
    uint32_t q;           /* 1-based label of the executed hop in its round */
    uint32_t p;           /* rounds used by this hop, including the accepting one */
    uint64_t round;       /* global round counter of the accepting round */
    int32_t dx, dy;       /* hop vector */
    double dE;            /* dH of the executed hop */
    uint32_t k, l;        /* second electron of a pair hop (R15); 0xFFFFFFFF otherwise */
    int32_t dx2, dy2;     /* its hop vector; 0 otherwise */
} orc_hop;

typedef struct orc_chain {
    int Lx, Ly, Lz, N, Hx, Hy, Hz;  /* Hx = Lx/2 + 1 folded extents */
    double nu, W, xi, T, E;
    int r_max;
    uint64_t seed;
    uint32_t replica;
    /* tables */
    double *tinv;             /* Hz x Hy x Hx, tinv[(fz*Hy + fy)*Hx + fx] = 1/r, 0 at 0 */
    int V;
    int32_t *vdx, *vdy, *vdz;
    double *w;                /* real tunnelling weights */
    uint64_t *Wint;           /* integer weights */
    uint64_t *C;              /* running sums */
    double Z;
    /* state */
    uint8_t *n;
    double *phi;
    double *eps;
    orc_counters cnt;
    int toy;                  /* test-only constant acceptance mode */
    double toy_A0;
    int time_mode;            /* 0: t = attempts / Gamma (R4); 1: Gaussian dt (R13) */
    uint32_t pair_T;          /* R15: pair proposal iff x3 < pair_T (0: single hops only) */
    int pair_R;               /* R15: pair offsets inside the disk |e| <= pair_R */
    /* R16: random sites */
    int random;               /* 1: sites at random positions (Lz = 1, Ly = Lx) */
    double *px, *py;          /* positions */
    int *roff;                /* N + 1 offsets of each site's partner list */
    uint32_t *rj;             /* partners */
    uint64_t *rC;             /* running integer weights within each list */
    double *rg, *rdx;         /* 1/r and the minimum-image x displacement of each pair */
    double Zmax;
} orc_chain;

static int fold(int d, int L)
{
    /* d in (-L, L): minimum-image |d| */
    int m = d % L;
    if (m < 0) m += L;
    return (m < L - m) ? m : L - m;
}

double orc_tinv_of3(const orc_chain *c, int dx, int dy, int dz)
{
    int fx = fold(dx, c->Lx), fy = fold(dy, c->Ly), fz = fold(dz, c->Lz);
    return c->tinv[(fz * c->Hy + fy) * c->Hx + fx];
}

double orc_tinv_of(const orc_chain *c, int dx, int dy)
{
    return orc_tinv_of3(c, dx, dy, 0);
}

/* R16: minimum-image displacement component from a to b in a box of side L */
static double min_image(double d, double L)
{
    if (d > 0.5 * L) d = d - L;
    else if (d < -0.5 * L) d = d + L;
    return d;
}

static double tinv_random(const orc_chain *c, int a, int b)
{
    double dx, dy;
    if (a == b) return 0.0;
    dx = min_image(c->px[b] - c->px[a], (double)c->Lx);
    dy = min_image(c->py[b] - c->py[a], (double)c->Lx);
    return 1.0 / sqrt(dx * dx + dy * dy);
}

/* site s = (z Ly + y) Lx + x */
static double tinv_sites(const orc_chain *c, int a, int b)
{
    if (c->random) return tinv_random(c, a, b);
    {
    int xa = a % c->Lx, ya = (a / c->Lx) % c->Ly, za = a / (c->Lx * c->Ly);
    int xb = b % c->Lx, yb = (b / c->Lx) % c->Ly, zb = b / (c->Lx * c->Ly);
    return orc_tinv_of3(c, xa - xb, ya - yb, za - zb);
    }
}

void orc_free(orc_chain *c)
{
    if (!c) return;
    free(c->tinv); free(c->vdx); free(c->vdy); free(c->vdz); free(c->w); free(c->Wint);
    free(c->C); free(c->n); free(c->phi); free(c->eps);
    free(c->px); free(c->py); free(c->roff); free(c->rj); free(c->rC); free(c->rg); free(c->rdx);
    free(c);
}

/* eps_s = phi_s + sum_{t != s} (n_t - nu) / r_st, summed over t = 0..N-1 in
 * increasing order, each product rounded before it is added (the summation
 * order the library's initial eps follows, so both give the same bits). */
void orc_eps_scratch(const orc_chain *c, double *out)
{
    int s, t;
    for (s = 0; s < c->N; ++s) {
        double acc = 0.0;
        for (t = 0; t < c->N; ++t) {
            double term;
            if (t == s) continue;
            term = ((double)c->n[t] - c->nu) * tinv_sites(c, s, t);
            acc = acc + term;
        }
        out[s] = c->phi[s] + acc;
    }
}

/* H of Eq. 1 from scratch, with the field term written with the site
 * coordinates x in [0, Lx).  Used for the initial energy only. */
double orc_energy_scratch(const orc_chain *c)
{
    double h1 = 0.0, h2 = 0.0, h3 = 0.0;
    int s, t;
    for (s = 0; s < c->N; ++s) {
        h1 = h1 + c->phi[s] * (double)c->n[s];
        /* the x position: the lattice column, or the random site's x (R16) */
        h3 = h3 + (double)c->n[s] * (c->random ? c->px[s] : (double)(s % c->Lx));
    }
    for (s = 0; s < c->N; ++s) {
        double ss = (double)c->n[s] - c->nu;
        for (t = 0; t < c->N; ++t) {
            if (t == s) continue;
            h2 = h2 + ss * ((double)c->n[t] - c->nu) * tinv_sites(c, s, t);
        }
    }
    return h1 + 0.5 * h2 - c->E * h3;
}

typedef struct { uint32_t key; uint32_t site; } orc_sortkey;

static int cmp_sortkey(const void *a, const void *b)
{
    const orc_sortkey *x = (const orc_sortkey *)a, *y = (const orc_sortkey *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->site != y->site) return x->site < y->site ? -1 : 1;
    return 0;
}

static void philox_setup_word(const orc_chain *c, uint32_t s, uint32_t domain,
                              uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = s; ctr[1] = domain; ctr[2] = 0xFFFFFFFFu; ctr[3] = c->replica;
    key[0] = (uint32_t)c->seed; key[1] = (uint32_t)(c->seed >> 32);
    orc_philox(ctr, key, out);
}

orc_chain *orc_new3(int Lx, int Ly, int Lz, double nu, double W, double xi, int r_max,
                    double T, double E, uint64_t seed, uint32_t replica)
{
    orc_chain *c;
    int fx, fy, fz, dx, dy, dz, k, s, nocc, Ry, Rz;
    double nuN;
    orc_sortkey *sk;

    if (Lx < 2 || Ly < 1 || Lz < 1 || (Lx % 2) || (Ly > 1 && (Ly % 2)) ||
        (Lz > 1 && (Lz % 2)) || (Lz > 1 && Ly == 1)) return NULL;
    if (!(nu > 0.0 && nu < 1.0) || !(xi > 0.0) || !(T > 0.0) || !(W >= 0.0)) return NULL;
    if (r_max < 1 || 2 * r_max >= Lx || (Ly > 1 && 2 * r_max >= Ly) ||
        (Lz > 1 && 2 * r_max >= Lz)) return NULL;
    nuN = nu * (double)(Lx * Ly * Lz);
    if (fabs(nuN - floor(nuN + 0.5)) > 1e-9) return NULL;

    c = (orc_chain *)calloc(1, sizeof(*c));
    if (!c) return NULL;
    c->Lx = Lx; c->Ly = Ly; c->Lz = Lz; c->N = Lx * Ly * Lz;
    c->Hx = Lx / 2 + 1; c->Hy = Ly / 2 + 1; c->Hz = Lz / 2 + 1;
    c->nu = nu; c->W = W; c->xi = xi; c->T = T; c->E = E; c->r_max = r_max;
    c->seed = seed; c->replica = replica;

    /* folded minimum-image 1/r table (reading R8: zero at the origin) */
    c->tinv = (double *)calloc((size_t)c->Hx * c->Hy * c->Hz, sizeof(double));
    for (fz = 0; fz < c->Hz; ++fz)
        for (fy = 0; fy < c->Hy; ++fy)
            for (fx = 0; fx < c->Hx; ++fx)
                c->tinv[(fz * c->Hy + fy) * c->Hx + fx] =
                    (fx == 0 && fy == 0 && fz == 0)
                        ? 0.0
                        : 1.0 / sqrt((double)(fx * fx + fy * fy + fz * fz));

    /* displacement list and tower (reading R2) */
    Ry = (Ly > 1) ? r_max : 0;
    Rz = (Lz > 1) ? r_max : 0;
    c->V = 0;
    for (dz = -Rz; dz <= Rz; ++dz)
        for (dy = -Ry; dy <= Ry; ++dy)
            for (dx = -r_max; dx <= r_max; ++dx) {
                int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > 0 && r2 <= r_max * r_max) c->V++;
            }
    c->vdx = (int32_t *)malloc(sizeof(int32_t) * c->V);
    c->vdy = (int32_t *)malloc(sizeof(int32_t) * c->V);
    c->vdz = (int32_t *)malloc(sizeof(int32_t) * c->V);
    c->w = (double *)malloc(sizeof(double) * c->V);
    c->Wint = (uint64_t *)malloc(sizeof(uint64_t) * c->V);
    c->C = (uint64_t *)malloc(sizeof(uint64_t) * c->V);
    k = 0;
    for (dz = -Rz; dz <= Rz; ++dz)
        for (dy = -Ry; dy <= Ry; ++dy)
            for (dx = -r_max; dx <= r_max; ++dx) {
                int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > 0 && r2 <= r_max * r_max) {
                    c->vdx[k] = dx; c->vdy[k] = dy; c->vdz[k] = dz;
                    c->w[k] = orc_exp_core(-2.0 * sqrt((double)r2) / xi);
                    ++k;
                }
            }
    c->Z = 0.0;
    for (k = 0; k < c->V; ++k) c->Z = c->Z + c->w[k];
    {
        uint64_t run = 0;
        for (k = 0; k < c->V; ++k) {
            double f = (c->w[k] / c->Z) * 4294967296.0;
            c->Wint[k] = (uint64_t)floor(f);
            run += c->Wint[k];
            c->C[k] = run;
        }
    }

    /* disorder (reading R5) */
    c->phi = (double *)malloc(sizeof(double) * c->N);
    c->n = (uint8_t *)calloc((size_t)c->N, 1);
    c->eps = (double *)malloc(sizeof(double) * c->N);
    for (s = 0; s < c->N; ++s) {
        uint32_t o[4];
        double u;
        philox_setup_word(c, (uint32_t)s, 1u, o);
        u = ((double)o[0] + 0.5) * 0x1p-32;
        c->phi[s] = W * (u - 0.5);
    }
    /* initial occupation (reading R6) */
    sk = (orc_sortkey *)malloc(sizeof(orc_sortkey) * c->N);
    for (s = 0; s < c->N; ++s) {
        uint32_t o[4];
        philox_setup_word(c, (uint32_t)s, 2u, o);
        sk[s].key = o[0];
        sk[s].site = (uint32_t)s;
    }
    qsort(sk, (size_t)c->N, sizeof(orc_sortkey), cmp_sortkey);
    nocc = (int)floor(nuN + 0.5);
    for (s = 0; s < nocc; ++s) c->n[sk[s].site] = 1;
    free(sk);

    orc_eps_scratch(c, c->eps);
    memset(&c->cnt, 0, sizeof(c->cnt));
    c->cnt.energy = orc_energy_scratch(c);
    {
        int64_t P = 0;
        for (s = 0; s < c->N; ++s) if (c->n[s]) P += s % c->Lx;
        c->cnt.P = P;
    }
    return c;
}

orc_chain *orc_new(int Lx, int Ly, double nu, double W, double xi, int r_max,
                   double T, double E, uint64_t seed, uint32_t replica)
{
    return orc_new3(Lx, Ly, 1, nu, W, xi, r_max, T, E, seed, replica);
}

/* R16: N = L^2 sites at random positions in the L x L periodic box.  The
 * lattice parts (disorder, initial state) are those of the L x L square
 * lattice; positions, partner lists and the tower follow the reading. */
orc_chain *orc_new_random(int L, double nu, double W, double xi, int r_max, double T,
                          double E, uint64_t seed, uint32_t replica)
{
    orc_chain *c = orc_new3(L, L, 1, nu, W, xi, r_max, T, E, seed, replica);
    int s, t, m, cnt;
    double *Z, *w;
    if (!c) return NULL;
    c->random = 1;
    c->px = (double *)malloc(sizeof(double) * c->N);
    c->py = (double *)malloc(sizeof(double) * c->N);
    for (s = 0; s < c->N; ++s) {
        uint32_t o[4];
        philox_setup_word(c, (uint32_t)s, 3u, o);
        c->px[s] = (double)L * (((double)o[0] + 0.5) * 0x1p-32);
        c->py[s] = (double)L * (((double)o[1] + 0.5) * 0x1p-32);
    }
    /* partner lists: count, then fill (ascending partner) */
    c->roff = (int *)calloc((size_t)c->N + 1, sizeof(int));
    cnt = 0;
    for (s = 0; s < c->N; ++s) {
        c->roff[s] = cnt;
        for (t = 0; t < c->N; ++t) {
            double dx, dy, r;
            if (t == s) continue;
            dx = min_image(c->px[t] - c->px[s], (double)L);
            dy = min_image(c->py[t] - c->py[s], (double)L);
            r = sqrt(dx * dx + dy * dy);
            if (r == 0.0) { orc_free(c); return NULL; }       /* coincident sites */
            if (r <= (double)r_max) ++cnt;
        }
    }
    c->roff[c->N] = cnt;
    c->rj = (uint32_t *)malloc(sizeof(uint32_t) * (cnt ? cnt : 1));
    c->rC = (uint64_t *)malloc(sizeof(uint64_t) * (cnt ? cnt : 1));
    c->rg = (double *)malloc(sizeof(double) * (cnt ? cnt : 1));
    c->rdx = (double *)malloc(sizeof(double) * (cnt ? cnt : 1));
    Z = (double *)calloc((size_t)c->N, sizeof(double));
    w = (double *)malloc(sizeof(double) * (cnt ? cnt : 1));
    m = 0;
    for (s = 0; s < c->N; ++s)
        for (t = 0; t < c->N; ++t) {
            double dx, dy, r;
            if (t == s) continue;
            dx = min_image(c->px[t] - c->px[s], (double)L);
            dy = min_image(c->py[t] - c->py[s], (double)L);
            r = sqrt(dx * dx + dy * dy);
            if (r > (double)r_max) continue;
            c->rj[m] = (uint32_t)t;
            c->rg[m] = 1.0 / r;
            c->rdx[m] = dx;
            w[m] = orc_exp_core(-2.0 * r / xi);
            Z[s] = Z[s] + w[m];
            ++m;
        }
    c->Zmax = 0.0;
    for (s = 0; s < c->N; ++s) if (Z[s] > c->Zmax) c->Zmax = Z[s];
    for (s = 0; s < c->N; ++s) {
        uint64_t run = 0;
        for (m = c->roff[s]; m < c->roff[s + 1]; ++m) {
            uint64_t Wm = (uint64_t)floor((w[m] / c->Zmax) * 4294967296.0);
            if (Wm > 0xFFFFFFFFull) Wm = 0xFFFFFFFFull;
            run += Wm;
            c->rC[m] = run;
        }
    }
    free(Z);
    free(w);
    /* eps, energy and the (untracked) dipole from scratch on the new geometry */
    orc_eps_scratch(c, c->eps);
    c->cnt.energy = orc_energy_scratch(c);
    c->cnt.P = 0;
    return c;
}

void orc_get_positions(const orc_chain *c, double *x, double *y)
{
    int s;
    for (s = 0; s < c->N; ++s) { x[s] = c->px[s]; y[s] = c->py[s]; }
}

int orc_num_pairs(const orc_chain *c) { return c->random ? c->roff[c->N] : 0; }

void orc_get_pairs(const orc_chain *c, int32_t *off, uint32_t *j, uint64_t *C, double *g,
                   double *dx)
{
    int s, m;
    for (s = 0; s <= c->N; ++s) off[s] = c->roff[s];
    for (m = 0; m < c->roff[c->N]; ++m) {
        j[m] = c->rj[m]; C[m] = c->rC[m]; g[m] = c->rg[m]; dx[m] = c->rdx[m];
    }
}

double orc_Zmax(const orc_chain *c) { return c->Zmax; }

/* ------------------------------------------------------------------------ */
/* Accessors                                                                 */
/* ------------------------------------------------------------------------ */

int orc_num_vectors(const orc_chain *c) { return c->V; }
int orc_num_sites(const orc_chain *c) { return c->N; }
double orc_Z(const orc_chain *c) { return c->Z; }
double orc_Gamma(const orc_chain *c)
{
    /* R4; with pair proposals (R15) a fraction T_p 2^-32 of the attempts is
       spent on them, so the single-hop attempts keep their rate */
    const double g = (double)c->N * (c->random ? c->Zmax : c->Z);
    return c->pair_T ? g / (1.0 - (double)c->pair_T * 0x1p-32) : g;
}

/* R15: pair proposals with probability p2 (0 <= p2 < 1) and offset radius R
 * (1 <= R, 2R below every side of the torus; square or cubic lattice). */
int orc_set_pair(orc_chain *c, double p2, int R)
{
    if (!(p2 >= 0.0 && p2 < 1.0)) return ORC_EINVAL;
    if (p2 > 0.0 && (c->random || c->Ly == 1 || R < 1 || 2 * R >= c->Lx || 2 * R >= c->Ly ||
                     (c->Lz > 1 && 2 * R >= c->Lz)))
        return ORC_EINVAL;
    c->pair_T = (uint32_t)floor(p2 * 4294967296.0);
    c->pair_R = p2 > 0.0 ? R : 0;
    return ORC_OK;
}

uint32_t orc_pair_threshold(const orc_chain *c) { return c->pair_T; }

void orc_get_vectors(const orc_chain *c, int32_t *dx, int32_t *dy,
                     uint64_t *Wint, double *w)
{
    int k;
    for (k = 0; k < c->V; ++k) {
        if (dx) dx[k] = c->vdx[k];
        if (dy) dy[k] = c->vdy[k];
        if (Wint) Wint[k] = c->Wint[k];
        if (w) w[k] = c->w[k];
    }
}

void orc_get_tinv(const orc_chain *c, double *out)
{
    memcpy(out, c->tinv, sizeof(double) * (size_t)c->Hx * c->Hy * c->Hz);
}

void orc_get_vectors_z(const orc_chain *c, int32_t *dz)
{
    int k;
    for (k = 0; k < c->V; ++k) dz[k] = c->vdz[k];
}

void orc_get_state(const orc_chain *c, uint8_t *n, double *eps, double *phi)
{
    if (n) memcpy(n, c->n, (size_t)c->N);
    if (eps) memcpy(eps, c->eps, sizeof(double) * c->N);
    if (phi) memcpy(phi, c->phi, sizeof(double) * c->N);
}

/* Replace occupation (and optionally disorder); eps is rebuilt from scratch,
 * the energy is recomputed from Eq. 1 and P from the coordinates. */
int orc_set_state(orc_chain *c, const uint8_t *n, const double *phi)
{
    int s;
    int64_t P = 0;
    for (s = 0; s < c->N; ++s) if (n[s] > 1) return ORC_EINVAL;
    memcpy(c->n, n, (size_t)c->N);
    if (phi) memcpy(c->phi, phi, sizeof(double) * c->N);
    orc_eps_scratch(c, c->eps);
    c->cnt.energy = orc_energy_scratch(c);
    for (s = 0; s < c->N; ++s) if (c->n[s]) P += s % c->Lx;
    c->cnt.P = P;
    return ORC_OK;
}

/* Overwrite eps directly (resume from a saved trajectory point). */
void orc_set_eps(orc_chain *c, const double *eps)
{
    memcpy(c->eps, eps, sizeof(double) * c->N);
}

void orc_get_counters(const orc_chain *c, orc_counters *out) { *out = c->cnt; }
void orc_set_counters(orc_chain *c, const orc_counters *in) { c->cnt = *in; }

void orc_set_time_mode(orc_chain *c, int mode) { c->time_mode = mode; }

void orc_set_toy(orc_chain *c, int on, double A0)
{
    c->toy = on;
    c->toy_A0 = A0;
}

/* dH of the hop i -> j with x-displacement dx, from the current eps (R9). */
double orc_delta_e(const orc_chain *c, int i, int j, int dx)
{
    double r_inv = tinv_sites(c, i, j);
    double d = c->eps[j] - c->eps[i];
    d = d - r_inv;
    return d - c->E * (double)dx;
}

/* dH of the pair hop i -> j, k -> l (x-displacements dx1, dx2) from the
 * current eps (R15): the two single-hop terms, then the interaction of the
 * second electron with the first one's move. */
double orc_delta_e_pair(const orc_chain *c, int i, int j, int k, int l, int dx1, int dx2)
{
    double d1 = orc_delta_e(c, i, j, dx1);
    double d2 = orc_delta_e(c, k, l, dx2);
    double cross = (tinv_sites(c, l, j) - tinv_sites(c, l, i)) -
                   (tinv_sites(c, k, j) - tinv_sites(c, k, i));
    return (d1 + d2) + cross;
}

/* ------------------------------------------------------------------------ */
/* One label: steps 1-2 of the mixed PR algorithm                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t accepted;
    int32_t vec;          /* displacement index, -1 for a null proposal */
    uint32_t i, j;
    int32_t dx, dy, dz;
    int32_t theta;        /* n_i = 1 and n_j = 0 (and the pair conditions of R15) */
    double dE;
    double u;
    uint32_t x[4];        /* raw Philox words */
    int32_t pair;         /* 1: a pair proposal (x3 < T_p, R15) */
    int32_t vec2;         /* its second vector, -1 for a null proposal */
    int32_t ex, ey, ez;   /* its offset e (ez = 0 on the square lattice) */
    uint32_t k, l;        /* its second electron's origin and destination */
    int32_t dx2, dy2, dz2;
    uint32_t y[4];        /* raw words of its second Philox block */
} orc_label;

static int tower_sample(const orc_chain *c, uint32_t x1)
{
    /* smallest k with x1 < C_k; -1 when x1 >= C_{V-1} (null proposal) */
    int lo = 0, hi = c->V;               /* answer in [lo, hi] */
    if ((uint64_t)x1 >= c->C[c->V - 1]) return -1;
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if ((uint64_t)x1 < c->C[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* The tower sampler for n words x1 (-1 marks a null proposal). */
void orc_tower_many(const orc_chain *c, const uint32_t *x1, int32_t *out, int n)
{
    int k;
    for (k = 0; k < n; ++k) out[k] = tower_sample(c, x1[k]);
}

void orc_eval_label(const orc_chain *c, uint64_t round, uint32_t k, orc_label *out)
{
    uint32_t ctr[4], key[2];
    int v, xi, yi, zi, xj, yj, zj;
    memset(out, 0, sizeof(*out));
    ctr[0] = k;
    ctr[1] = (uint32_t)round;
    ctr[2] = (uint32_t)(round >> 32);
    ctr[3] = c->replica;
    key[0] = (uint32_t)c->seed;
    key[1] = (uint32_t)(c->seed >> 32);
    orc_philox(ctr, key, out->x);

    out->i = (uint32_t)(((uint64_t)out->x[0] * (uint64_t)c->N) >> 32);
    out->u = ((double)out->x[2] + 0.5) * 0x1p-32;
    out->pair = out->x[3] < c->pair_T;       /* R15 */
    if (c->random && !c->toy) {
        /* R16: the partner of i by the integer tower of i's list */
        int m, lo = c->roff[out->i], hi = c->roff[out->i + 1];
        out->vec = -1;
        for (m = lo; m < hi; ++m)
            if ((uint64_t)out->x[1] < c->rC[m]) { out->vec = m; break; }
        if (out->vec < 0) { out->accepted = 0; return; }
        out->j = c->rj[out->vec];
        out->theta = (c->n[out->i] == 1) && (c->n[out->j] == 0);
        if (!out->theta) { out->accepted = 0; return; }
        out->dE = ((c->eps[out->j] - c->eps[out->i]) - c->rg[out->vec]) -
                  c->E * c->rdx[out->vec];
        if (out->dE <= 0.0) { out->accepted = 1; return; }
        out->accepted = out->u < orc_cg_exp((-out->dE) / c->T);
        return;
    }
    v = tower_sample(c, out->x[1]);
    out->vec = v;
    if (c->toy) {                        /* test-only: constant acceptance */
        out->accepted = out->u < c->toy_A0;
        return;
    }
    if (v < 0) { out->accepted = 0; return; }
    out->dx = c->vdx[v];
    out->dy = c->vdy[v];
    out->dz = c->vdz[v];
    xi = (int)(out->i % (uint32_t)c->Lx);
    yi = (int)((out->i / (uint32_t)c->Lx) % (uint32_t)c->Ly);
    zi = (int)(out->i / (uint32_t)(c->Lx * c->Ly));
    xj = (xi + out->dx + c->Lx) % c->Lx;
    yj = (yi + out->dy + c->Ly) % c->Ly;
    zj = (zi + out->dz + c->Lz) % c->Lz;
    out->j = (uint32_t)((zj * c->Ly + yj) * c->Lx + xj);
    out->theta = (c->n[out->i] == 1) && (c->n[out->j] == 0);
    out->k = 0xFFFFFFFFu;
    out->l = 0xFFFFFFFFu;
    if (out->pair) {
        /* R15: a pair proposal */
        int R = c->pair_R, W = 2 * c->pair_R + 1, xk, yk, zk, xl, yl, zl, fx, fy, fz, e2, f2;
        ctr[2] = (uint32_t)(round >> 32) | 0x80000000u;
        orc_philox(ctr, key, out->y);
        out->ex = (int)(((uint64_t)out->y[0] * (uint64_t)W) >> 32) - R;
        out->ey = (int)(((uint64_t)out->y[2] * (uint64_t)W) >> 32) - R;
        /* on the cubic lattice the offset's z comes from the fourth word */
        out->ez = c->Lz > 1 ? (int)(((uint64_t)out->y[3] * (uint64_t)W) >> 32) - R : 0;
        out->vec2 = tower_sample(c, out->y[1]);
        if (out->vec2 < 0) { out->theta = 0; out->accepted = 0; return; }
        out->dx2 = c->vdx[out->vec2];
        out->dy2 = c->vdy[out->vec2];
        out->dz2 = c->vdz[out->vec2];
        xk = (xi + out->ex + c->Lx) % c->Lx;
        yk = (yi + out->ey + c->Ly) % c->Ly;
        zk = (zi + out->ez + c->Lz) % c->Lz;
        xl = (xk + out->dx2 + c->Lx) % c->Lx;
        yl = (yk + out->dy2 + c->Ly) % c->Ly;
        zl = (zk + out->dz2 + c->Lz) % c->Lz;
        out->k = (uint32_t)((zk * c->Ly + yk) * c->Lx + xk);
        out->l = (uint32_t)((zl * c->Ly + yl) * c->Lx + xl);
        fx = out->ex + out->dx2 - out->dx;          /* e' = l - j */
        fy = out->ey + out->dy2 - out->dy;
        fz = out->ez + out->dz2 - out->dz;
        e2 = out->ex * out->ex + out->ey * out->ey + out->ez * out->ez;
        f2 = fx * fx + fy * fy + fz * fz;
        out->theta = out->theta && c->n[out->k] == 1 && c->n[out->l] == 0 &&
                     e2 > 0 && e2 <= R * R && f2 > 0 && f2 <= R * R;
        if (!out->theta) { out->accepted = 0; return; }
        out->dE = orc_delta_e_pair(c, (int)out->i, (int)out->j, (int)out->k, (int)out->l,
                                   out->dx, out->dx2);
    } else {
        if (!out->theta) { out->accepted = 0; return; }
        out->dE = orc_delta_e(c, (int)out->i, (int)out->j, out->dx);
    }
    if (out->dE <= 0.0) { out->accepted = 1; return; }
    out->accepted = out->u < orc_cg_exp((-out->dE) / c->T);
}

/* ------------------------------------------------------------------------ */
/* Step 3: execute the hop                                                   */
/* ------------------------------------------------------------------------ */

static void commit_hop(orc_chain *c, const orc_label *lab)
{
    int l;
    uint32_t i = lab->i, j = lab->j;
    if (c->toy) return;                  /* toy mode moves no electron */
    c->n[i] = 0;
    c->n[j] = 1;
    if (!c->random) c->cnt.P += lab->dx;        /* R16: no dipole on random sites */
    c->cnt.energy = c->cnt.energy + lab->dE;
    for (l = 0; l < c->N; ++l) {
        double delta = tinv_sites(c, l, (int)j) - tinv_sites(c, l, (int)i);
        c->eps[l] = c->eps[l] + delta;
    }
    if (lab->pair) {
        /* R15: the second electron's move, applied after the first one's */
        uint32_t k = lab->k, m = lab->l;
        c->n[k] = 0;
        c->n[m] = 1;
        c->cnt.P += lab->dx2;
        for (l = 0; l < c->N; ++l) {
            double delta = tinv_sites(c, l, (int)m) - tinv_sites(c, l, (int)k);
            c->eps[l] = c->eps[l] + delta;
        }
    }
}

/* Run until n_hops more hops are executed.  M labels per round; a hop whose
 * rounds reach max_rounds without an accept ends the call with ORC_ESTUCK
 * (the failed rounds are counted).  log, when given, receives one entry per
 * executed hop. */
int orc_run(orc_chain *c, uint64_t n_hops, uint32_t M, uint64_t max_rounds,
            orc_hop *log)
{
    uint64_t h;
    if (M == 0) return ORC_EINVAL;
    for (h = 0; h < n_hops; ++h) {
        uint32_t p = 0;
        for (;;) {
            uint32_t k;
            int done = 0;
            orc_label lab;
            ++p;
            for (k = 0; k < M; ++k) {
                orc_eval_label(c, c->cnt.rounds, k, &lab);
                c->cnt.evaluated++;
                if (lab.accepted) { done = 1; break; }
            }
            if (done) {
                uint32_t q = k + 1;
                if (log) {
                    orc_hop *e = &log[h];
                    e->i = lab.i; e->j = lab.j; e->q = q; e->p = p;
                    e->round = c->cnt.rounds;
                    e->dx = lab.dx; e->dy = lab.dy; e->dE = lab.dE;
                    e->k = lab.pair ? lab.k : 0xFFFFFFFFu;
                    e->l = lab.pair ? lab.l : 0xFFFFFFFFu;
                    e->dx2 = lab.pair ? lab.dx2 : 0;
                    e->dy2 = lab.pair ? lab.dy2 : 0;
                }
                if (c->time_mode) {
                    uint64_t m = (uint64_t)(p - 1) * M + q;
                    double z = orc_gauss(c->seed, c->replica, c->cnt.hops);
                    c->cnt.time = c->cnt.time + orc_time_increment(orc_Gamma(c), m, z);
                }
                c->cnt.attempts += q;
                c->cnt.rounds += 1;
                c->cnt.hops += 1;
                commit_hop(c, &lab);
                break;
            }
            c->cnt.attempts += M;
            c->cnt.rounds += 1;
            if ((uint64_t)p >= max_rounds) return ORC_ESTUCK;
        }
    }
    return ORC_OK;
}
