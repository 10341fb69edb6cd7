// cg_refresh_fft.cu -- the binary32 refresh of eps from its definition below
// Eq. 2 by the convolution theorem.  On the periodic lattice
//     eps_s - phi_s = sum_t g(s - t) (n_t - nu),
// g the minimum-image 1/r with g(0) = 0, is a circular convolution, so
// eps - phi = IDFT(DFT(n - nu) . DFT(g)).  g is even, so DFT(g) is real and
// two replicas share one complex transform: z = a + i b (a, b = n - nu of the
// two) gives IDFT(DFT(z) . DFT(g)) = (a * g) + i (b * g).
//
// L = 2^m or 3 2^m.  Transforms in binary32 along one axis per pass, W lines
// per CTA in shared memory.  L = 2^m: a forward pass loads in bit-reversed
// order and runs radix-2 decimation-in-time butterflies (natural-order
// output); an inverse pass runs decimation-in-frequency butterflies on
// natural-order input and stores from the bit-reversed positions.  L = 3M
// (M = 2^m), both directions: with n = M n1 + n2 and k = k1 + 3 k2,
//     X[k1 + 3 k2] = sum_n2 W_M^(n2 k2) W_L^(n2 k1) sum_n1 W_3^(n1 k1) x[M n1 + n2],
// a radix-3 step over the thirds of the line with the twiddles W_L^(n2 k1),
// then an M-point decimation-in-frequency transform of each third; X[k]
// sits at (k mod 3) M + bitrev(k / 3).  Passes:
//   square lattice: forward x (from the bitmasks) | forward y, times
//                   DFT(g)/N, inverse y | inverse x (into eps);
//   cubic lattice:  forward x | forward y | forward z, times DFT(g)/N,
//                   inverse z | inverse y | inverse x (into eps).
// The last pass adds phi in binary64, stores eps rounded to binary32 and
// records the largest |eps_old - eps_new| of each replica, as the other
// refresh paths do.  The product's table DFT(g)/N and the twiddles
// exp(-2 pi i k / L) are computed on the host in binary64.
#include "cg_device.cuh"
#include "cg_internal.h"

namespace cg {

namespace {

constexpr int kFftThreads = 256;

struct FftArgs {
    const DevReplica *reps;
    const int *index;     // the group's replicas, in group order
    int R, L, log2L, W;   // replicas; side (log2L: of a power-of-two L); lines per CTA
    int M3, log2M;        // L = 3 M3 (0 for a power-of-two L), log2 M3
    float2 *buf;          // ceil(R/2) x N complex values
    const float *ghat;    // N: DFT(g) / N
    const float2 *tw;     // L: exp(-2 pi i k / L)
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ unsigned bitrev(unsigned k, int log2L)
{
    return __brev(k) >> (32 - log2L);
}

// Element (w, k) of line group g of pair p along `axis`: its site index.
// axis 0: rows g W + w, element k along x; axis 1: z = g / (L/W), columns
// x0 + w, element k along y; axis 2: y = g / (L/W), columns x0 + w,
// element k along z.
__device__ __forceinline__ unsigned site_of(int axis, int g, int w, int k, int L, int W)
{
    if (axis == 0) return (unsigned)((g * W + w) * L + k);
    const int per = L / W;
    const int o = g / per, x0 = (g - o * per) * W;
    if (axis == 1) return (unsigned)((o * L + k) * L + x0 + w);
    return (unsigned)((k * L + o) * L + x0 + w);
}

// Radix-2 decimation in time on W lines of length L in shared memory (line
// stride Ls), input in bit-reversed order; conj: the inverse transform.
__device__ __forceinline__ void dit(float2 *s, int Ls, const FftArgs &a, bool conj)
{
    const int L = a.L, half = L >> 1, nb = a.W * half;
    for (int st = 0; st < a.log2L; ++st) {
        const int h = 1 << st;
        for (int b = threadIdx.x; b < nb; b += kFftThreads) {
            const int w = b >> (a.log2L - 1), j = b & (half - 1);
            const int pos = j & (h - 1), i0 = ((j >> st) << (st + 1)) + pos, i1 = i0 + h;
            float2 t = a.tw[pos << (a.log2L - 1 - st)];
            if (conj) t.y = -t.y;
            float2 *l = s + w * Ls;
            const float2 x0 = l[i0], u = cmul(l[i1], t);
            l[i0] = make_float2(x0.x + u.x, x0.y + u.y);
            l[i1] = make_float2(x0.x - u.x, x0.y - u.y);
        }
        __syncthreads();
    }
}

// Radix-2 decimation in frequency, natural-order input, bit-reversed output.
__device__ __forceinline__ void dif(float2 *s, int Ls, const FftArgs &a, bool conj)
{
    const int L = a.L, half = L >> 1, nb = a.W * half;
    for (int st = a.log2L - 1; st >= 0; --st) {
        const int h = 1 << st;
        for (int b = threadIdx.x; b < nb; b += kFftThreads) {
            const int w = b >> (a.log2L - 1), j = b & (half - 1);
            const int pos = j & (h - 1), i0 = ((j >> st) << (st + 1)) + pos, i1 = i0 + h;
            float2 t = a.tw[pos << (a.log2L - 1 - st)];
            if (conj) t.y = -t.y;
            float2 *l = s + w * Ls;
            const float2 x0 = l[i0], x1 = l[i1];
            l[i0] = make_float2(x0.x + x1.x, x0.y + x1.y);
            l[i1] = cmul(make_float2(x0.x - x1.x, x0.y - x1.y), t);
        }
        __syncthreads();
    }
}

// L = 3 M: the radix-3 step with its twiddles, then an M-point
// decimation-in-frequency transform of each third (natural-order input;
// X[k] at (k mod 3) M + bitrev(k / 3)).  conj: the inverse transform.
__device__ __forceinline__ void mixed3(float2 *s, int Ls, const FftArgs &a, bool conj)
{
    const int M = a.M3, lm = a.log2M, nb3 = a.W * M;
    const float c = 0.8660254037844386f;                  // sqrt(3) / 2
    for (int b = threadIdx.x; b < nb3; b += kFftThreads) {
        const int w = b >> lm, n2 = b & (M - 1);
        float2 *l = s + w * Ls;
        const float2 x0 = l[n2], x1 = l[M + n2], x2 = l[2 * M + n2];
        const float2 s1 = make_float2(x1.x + x2.x, x1.y + x2.y);
        const float2 d1 = make_float2(x1.x - x2.x, x1.y - x2.y);
        const float2 t = make_float2(fmaf(-0.5f, s1.x, x0.x), fmaf(-0.5f, s1.y, x0.y));
        const float sg = conj ? -1.0f : 1.0f;
        float2 y1 = make_float2(fmaf(sg * c, d1.y, t.x), fmaf(-sg * c, d1.x, t.y));
        float2 y2 = make_float2(fmaf(-sg * c, d1.y, t.x), fmaf(sg * c, d1.x, t.y));
        float2 w1 = a.tw[n2], w2 = a.tw[2 * n2];
        if (conj) {
            w1.y = -w1.y;
            w2.y = -w2.y;
        }
        l[n2] = make_float2(x0.x + s1.x, x0.y + s1.y);
        l[M + n2] = cmul(y1, w1);
        l[2 * M + n2] = cmul(y2, w2);
    }
    __syncthreads();
    const int half = M >> 1, nb = a.W * 3 * half;
    for (int st = lm - 1; st >= 0; --st) {
        const int h = 1 << st;
        for (int b = threadIdx.x; b < nb; b += kFftThreads) {
            const int sub = b >> (lm - 1), j = b & (half - 1);
            const int w = sub / 3, k1 = sub - 3 * w;
            const int pos = j & (h - 1), i0 = ((j >> st) << (st + 1)) + pos, i1 = i0 + h;
            float2 t = a.tw[3 * (pos << (lm - 1 - st))];        // W_M^(pos M / 2h)
            if (conj) t.y = -t.y;
            float2 *l = s + w * Ls + k1 * M;
            const float2 x0 = l[i0], x1 = l[i1];
            l[i0] = make_float2(x0.x + x1.x, x0.y + x1.y);
            l[i1] = cmul(make_float2(x0.x - x1.x, x0.y - x1.y), t);
        }
        __syncthreads();
    }
}

// Position in the line of output element k after a transform: L = 3 M
// (either direction), or L = 2^m after the inverse (decimation in frequency).
__device__ __forceinline__ int out_pos(int k, const FftArgs &a, bool dif_out)
{
    if (a.M3) {
        const int k2 = k / 3;
        return (k - 3 * k2) * a.M3 + (int)bitrev((unsigned)k2, a.log2M);
    }
    return dif_out ? (int)bitrev((unsigned)k, a.log2L) : k;
}

// One pass over W lines of one pair.  kMode: 0 forward x from the bitmasks;
// 1 forward (buffer to buffer); 2 forward, product with DFT(g)/N, inverse
// (the last axis); 3 inverse (buffer to buffer); 4 inverse x into eps.
// grid.x = pairs x line groups per pair.
template <int kMode>
__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(FftArgs a, int axis)
{
    extern __shared__ float2 s[];
    __shared__ unsigned long long s_err[2];
    const int L = a.L, W = a.W, Ls = L + 1;     // padded line stride (banks)
    const int groups = (int)(gridDim.x / (unsigned)((a.R + 1) / 2));
    const int p = blockIdx.x / groups, g = blockIdx.x - p * groups;
    const DevReplica &Ra = a.reps[a.index[2 * p]];
    const bool two = 2 * p + 1 < a.R;
    const DevReplica &Rb = a.reps[a.index[two ? 2 * p + 1 : 2 * p]];
    const unsigned Nr = (unsigned)Ra.N;                    // L^2 or L^3
    float2 *buf = a.buf + (size_t)p * Nr;
    const int n = W * L;
    const bool mixed = a.M3 != 0;
    // natural-order load for the inverse and for every L = 3 M transform
    const bool natural_in = kMode >= 3 || mixed;
    // ---- load ----
    for (int e = threadIdx.x; e < n; e += kFftThreads) {
        int w, k;
        if (axis == 0) { w = e / L; k = e - w * L; } else { k = e / W; w = e - k * W; }
        const unsigned site = site_of(axis, g, w, k, L, W);
        float2 v;
        if (kMode == 0) {
            const float na = (float)((Ra.occ[site >> 5] >> (site & 31)) & 1u) - (float)Ra.nu;
            const float nb = two ? (float)((Rb.occ[site >> 5] >> (site & 31)) & 1u) - (float)Rb.nu
                                 : 0.0f;
            v = make_float2(na, nb);
        } else {
            v = buf[site];
        }
        s[w * Ls + (natural_in ? k : (int)bitrev((unsigned)k, a.log2L))] = v;
    }
    if (kMode == 4 && threadIdx.x < 2) s_err[threadIdx.x] = 0ull;
    __syncthreads();
    // ---- transform ----
    float2 *out = s;                                       // where the result lies
    if (!mixed) {
        if (kMode <= 2) dit(s, Ls, a, false);
        if (kMode == 2) {
            for (int e = threadIdx.x; e < n; e += kFftThreads) {
                int w, k;
                if (axis == 0) { w = e / L; k = e - w * L; } else { k = e / W; w = e - k * W; }
                const float gh = a.ghat[site_of(axis, g, w, k, L, W)];
                float2 &v = s[w * Ls + k];
                v = make_float2(v.x * gh, v.y * gh);
            }
            __syncthreads();
        }
        if (kMode >= 2) dif(s, Ls, a, true);
    } else {
        mixed3(s, Ls, a, kMode >= 3);
        if (kMode == 2) {
            // the product in natural order into the second buffer, then the
            // inverse transform there
            float2 *s2 = s + W * Ls;
            for (int e = threadIdx.x; e < n; e += kFftThreads) {
                int w, k;
                if (axis == 0) { w = e / L; k = e - w * L; } else { k = e / W; w = e - k * W; }
                const float gh = a.ghat[site_of(axis, g, w, k, L, W)];
                const float2 v = s[w * Ls + out_pos(k, a, false)];
                s2[w * Ls + k] = make_float2(v.x * gh, v.y * gh);
            }
            __syncthreads();
            mixed3(s2, Ls, a, true);
            out = s2;
        }
    }
    // ---- store ----
    double err_a = 0.0, err_b = 0.0;
    if (kMode != 4) {
        for (int e = threadIdx.x; e < n; e += kFftThreads) {
            int w, k;
            if (axis == 0) { w = e / L; k = e - w * L; } else { k = e / W; w = e - k * W; }
            const unsigned site = site_of(axis, g, w, k, L, W);
            buf[site] = out[w * Ls + out_pos(k, a, kMode >= 2)];
        }
    } else {
        // axis x: element e of the CTA is site g W L + e.  phi and eps of
        // different sites are independent, so four elements' loads are in
        // flight at once (restrict: eps is not phi)
        const unsigned site0 = (unsigned)(g * W) * (unsigned)L;
        const double *__restrict__ pa = Ra.phi + site0;
        const double *__restrict__ pb = Rb.phi + site0;
        float *__restrict__ ea = reinterpret_cast<float *>(Ra.eps) + site0;
        float *__restrict__ eb = reinterpret_cast<float *>(Rb.eps) + site0;
        // the transforms took n - nu with nu rounded to binary32; sum_t g(s-t)
        // = C0 for every s, so (nu_f - nu) C0 restores the exact nu
        const double ca = d_mul(d_sub((double)(float)Ra.nu, Ra.nu), Ra.C0);
        const double cb = d_mul(d_sub((double)(float)Rb.nu, Rb.nu), Rb.C0);
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += kFftThreads) {
            const int w = e / L, k = e - w * L;
            const float2 v = out[w * Ls + out_pos(k, a, true)];
            const double na = d_add(pa[e], d_add((double)v.x, ca));
            err_a = fmax(err_a, fabs((double)ea[e] - na));
            ea[e] = __double2float_rn(na);
            if (two) {
                const double nb = d_add(pb[e], d_add((double)v.y, cb));
                err_b = fmax(err_b, fabs((double)eb[e] - nb));
                eb[e] = __double2float_rn(nb);
            }
        }
    }
    if (kMode == 4) {
        // block maxima of the non-negative errors through their bit patterns
        unsigned long long ba = (unsigned long long)__double_as_longlong(err_a);
        unsigned long long bb = (unsigned long long)__double_as_longlong(err_b);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long xa = __shfl_xor_sync(0xffffffffu, ba, o);
            const unsigned long long xb = __shfl_xor_sync(0xffffffffu, bb, o);
            ba = ba > xa ? ba : xa;
            bb = bb > xb ? bb : xb;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&s_err[0], ba);
            atomicMax(&s_err[1], bb);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicMax(&Ra.ctr->max_err_bits, s_err[0]);
            if (g == 0) atomicAdd(&Ra.ctr->refreshes, 1ull);
            if (two) {
                atomicMax(&Rb.ctr->max_err_bits, s_err[1]);
                if (g == 0) atomicAdd(&Rb.ctr->refreshes, 1ull);
            }
        }
    }
}

template <int kMode>
cudaError_t launch_pass(const FftArgs &a, int axis, int pairs, int groups, cudaStream_t st)
{
    // L = 3 M: the middle pass keeps a second buffer for the product
    const int smem = (a.M3 && kMode == 2 ? 2 : 1) * a.W * (a.L + 1) * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel<kMode>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    fft_pass_kernel<kMode><<<pairs * groups, kFftThreads, smem, st>>>(a, axis);
    return cudaGetLastError();
}

}  // namespace

// lines per CTA: the largest power of two up to 16 that divides L (the y and
// z passes take W adjacent columns) with W L <= 8192 values of shared memory
static int refresh_fft_lines(int L)
{
    int W = 16;
    while (W > 1 && (L % W != 0 || W * L > 8192)) W >>= 1;
    return W;
}

// The sides the FFT refresh takes: 2^m (4 <= L <= 1024) or 3 2^m (6 <= L <= 192).
bool refresh_fft_size_ok(int L)
{
    if (L >= 4 && L <= 1024 && (L & (L - 1)) == 0) return true;
    const int M = L / 3;
    return L % 3 == 0 && L >= 6 && L <= 192 && (M & (M - 1)) == 0;
}

cudaError_t launch_refresh_fft(const DevReplica *d_reps, const int *d_index, int R, int L,
                               int dim, const float *d_ghat, const float2 *d_tw, float2 *d_buf,
                               cudaStream_t st)
{
    if (R < 1 || !refresh_fft_size_ok(L) || (dim != 2 && dim != 3)) return cudaErrorInvalidValue;
    FftArgs a;
    a.reps = d_reps;
    a.index = d_index;
    a.R = R;
    a.L = L;
    const bool pow2 = (L & (L - 1)) == 0;
    a.log2L = pow2 ? __builtin_ctz((unsigned)L) : 0;
    a.M3 = pow2 ? 0 : L / 3;
    a.log2M = pow2 ? 0 : __builtin_ctz((unsigned)(L / 3));
    a.W = refresh_fft_lines(L);
    a.buf = d_buf;
    a.ghat = d_ghat;
    a.tw = d_tw;
    const int pairs = (R + 1) / 2;
    const int lines = dim == 3 ? L * L : L;              // lines per axis per pair
    const int groups = lines / a.W;
    cudaError_t e;
    if (dim == 2) {
        if ((e = launch_pass<0>(a, 0, pairs, groups, st))) return e;
        if ((e = launch_pass<2>(a, 1, pairs, groups, st))) return e;
        return launch_pass<4>(a, 0, pairs, groups, st);
    }
    if ((e = launch_pass<0>(a, 0, pairs, groups, st))) return e;
    if ((e = launch_pass<1>(a, 1, pairs, groups, st))) return e;
    if ((e = launch_pass<2>(a, 2, pairs, groups, st))) return e;
    if ((e = launch_pass<3>(a, 1, pairs, groups, st))) return e;
    return launch_pass<4>(a, 0, pairs, groups, st);
}

size_t refresh_fft_buffer_bytes(int N, int R) { return (size_t)((R + 1) / 2) * (size_t)N * 8; }

}  // namespace cg
