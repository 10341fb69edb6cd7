// cg_refresh_fft.cu -- the binary32 refresh of eps from its definition below
// Eq. 2 by the convolution theorem.  On the periodic lattice
//     eps_s - phi_s = sum_t g(s - t) (n_t - nu),
// g the minimum-image 1/r with g(0) = 0, is a circular convolution, so
// eps - phi = IDFT(DFT(n - nu) . DFT(g)).  g is even, so DFT(g) is real and
// two replicas share one complex transform: z = a + i b (a, b = n - nu of the
// two) gives IDFT(DFT(z) . DFT(g)) = (a * g) + i (b * g).
//
// Power-of-two L.  Radix-2 transforms in binary32 along one axis per pass,
// W lines per CTA in shared memory: a forward pass loads in bit-reversed
// order and runs decimation-in-time butterflies (natural-order output); an
// inverse pass runs decimation-in-frequency butterflies on natural-order
// input and stores from the bit-reversed positions.  Passes:
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
    int R, L, log2L, W;   // replicas; side; lines per CTA
    float2 *buf;          // ceil(R/2) x N complex values
    const float *ghat;    // N: DFT(g) / N
    const float2 *tw;     // L/2: exp(-2 pi i k / L)
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
    const bool inverse_in = kMode >= 3;                    // natural-order load
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
        s[w * Ls + (inverse_in ? k : (int)bitrev((unsigned)k, a.log2L))] = v;
    }
    if (kMode == 4 && threadIdx.x < 2) s_err[threadIdx.x] = 0ull;
    __syncthreads();
    // ---- transform ----
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
    // ---- store ----
    double err_a = 0.0, err_b = 0.0;
    if (kMode != 4) {
        for (int e = threadIdx.x; e < n; e += kFftThreads) {
            int w, k;
            if (axis == 0) { w = e / L; k = e - w * L; } else { k = e / W; w = e - k * W; }
            const unsigned site = site_of(axis, g, w, k, L, W);
            buf[site] = s[w * Ls + (kMode >= 2 ? (int)bitrev((unsigned)k, a.log2L) : k)];
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
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += kFftThreads) {
            const int w = e / L, k = e - w * L;
            const float2 v = s[w * Ls + (int)bitrev((unsigned)k, a.log2L)];
            const double na = d_add(pa[e], (double)v.x);
            err_a = fmax(err_a, fabs((double)ea[e] - na));
            ea[e] = __double2float_rn(na);
            if (two) {
                const double nb = d_add(pb[e], (double)v.y);
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
    const int smem = a.W * (a.L + 1) * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel<kMode>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    fft_pass_kernel<kMode><<<pairs * groups, kFftThreads, smem, st>>>(a, axis);
    return cudaGetLastError();
}

}  // namespace

// lines per CTA: 16, fewer where L is large (at most 8192 values of shared
// memory) or small (the y and z passes take W adjacent columns)
static int refresh_fft_lines(int L) { return L >= 16 ? (8192 / L < 16 ? 8192 / L : 16) : L; }

cudaError_t launch_refresh_fft(const DevReplica *d_reps, const int *d_index, int R, int L,
                               int dim, const float *d_ghat, const float2 *d_tw, float2 *d_buf,
                               cudaStream_t st)
{
    if (R < 1 || L < 4 || (L & (L - 1)) != 0 || L > 1024 || (dim != 2 && dim != 3))
        return cudaErrorInvalidValue;
    FftArgs a;
    a.reps = d_reps;
    a.index = d_index;
    a.R = R;
    a.L = L;
    a.log2L = __builtin_ctz((unsigned)L);
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
