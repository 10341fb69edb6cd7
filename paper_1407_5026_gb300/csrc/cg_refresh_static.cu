// cg_refresh_static.cu -- the tensor-core eps refresh for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs inside a host program which owns the device
// allocator (a framework with its own memory pool, or a rule that only the
// host program may allocate), a service that must not grow its device
// footprint after start-up, and code that must not make an allocation call at
// all on its hot path.  cg_refresh_tc_noalloc runs the same three refresh
// kernels as cg_refresh (S image, split-BF16 tcgen05 contraction, binary64
// reduction) on inputs and outputs the caller owns, and takes every piece of
// scratch -- replica descriptors, counters, the split 1/r table, the +-1
// occupation image and the K-split partial sums -- from one file-scope device
// array of kStaticScratchBytes.  That array exists on every GPU that loads the
// library and stays there until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda.h>   // CUcontext / CUresult types of two driver entry points

#include "cg_device.cuh"
#include "cg_internal.h"

namespace cg {

void set_last_error(const std::string &msg);   // cg_lib.cu

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

// The scratch of every call.  In host code this name is only a stand-in for
// the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_refresh_scratch[kStaticScratchBytes];

std::mutex g_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context id the address belongs to

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Unique id of the CUDA context current on this thread (cuCtxGetCurrent +
// cuCtxGetId through the runtime's driver entry points), 0 when there is none
// or it cannot be read.  A device address of the static array is valid only in
// the context it was looked up in: after cudaDeviceReset, or under another
// context on the same ordinal, the array lives elsewhere.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx &&
        get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the static scratch on the current device: looked up with
// that device current, once per device and context (again when the context
// changed, e.g. after cudaDeviceReset).
int scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_last_error("device ordinal out of range");
        return CG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_refresh_scratch);
        if (e != cudaSuccess) {
            set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return CG_ECUDA;
        }
        g_scratch_ptr[device] = static_cast<unsigned char *>(p);
        // the lookup makes the device's context current if none was
        g_scratch_ctx[device] = current_context_id();
    }
    *out = g_scratch_ptr[device];
    return CG_OK;
}

__device__ __forceinline__ uint32_t bf16_rne_dev(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}

// Descriptors of the caller's replica-major arrays, counters cleared, error
// word cleared.
__global__ void static_setup_kernel(DevReplica *reps, int *index, DevCounters *ctr, int *err,
                                    int R, int L, double nu, double C0,
                                    const unsigned int *occ, const double *phi, float *eps)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) *err = 0;
    if (r >= R) return;
    const int N = L * L, words = (N + 31) / 32;
    DevCounters c;
    memset(&c, 0, sizeof(c));
    ctr[r] = c;
    DevReplica d;
    memset(&d, 0, sizeof(d));
    d.L = L;
    d.N = N;
    d.H1 = L / 2 + 1;
    d.words = words;
    d.magicL = (unsigned)(4294967296ull / (unsigned long long)L + 1ull);
    d.nu = nu;
    d.C0 = C0;
    d.eps = eps + (size_t)r * N;
    d.occ = const_cast<unsigned int *>(occ) + (size_t)r * words;
    d.phi = phi + (size_t)r * N;
    d.ctr = ctr + r;
    reps[r] = d;
    index[r] = r;
}

// BF16 hi | lo << 16 of the folded 1/r table, the same split as the handle's
// table (hi = bf16(binary32(T)), lo = bf16(binary32(T - hi))).
__global__ void static_split_table_kernel(uint32_t *tab, int L)
{
    const int H1 = L / 2 + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= H1 * H1) return;
    const int fy = k / H1, fx = k - fy * H1;
    const double T = (fx == 0 && fy == 0)
                         ? 0.0
                         : __ddiv_rn(1.0, __dsqrt_rn((double)(fx * fx + fy * fy)));
    const uint32_t hi = bf16_rne_dev(__double2float_rn(T));
    const double rest = __dsub_rn(T, (double)__uint_as_float(hi << 16));
    const uint32_t lo = bf16_rne_dev(__double2float_rn(rest));
    tab[k] = hi | (lo << 16);
}

__global__ void static_err_out_kernel(const DevCounters *ctr, double *max_err, int R)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) max_err[r] = __longlong_as_double((long long)ctr[r].max_err_bits);
}

}  // namespace

// Bytes of static scratch a call with these sizes uses.
size_t noalloc_scratch_bytes(int L, int R)
{
    const size_t H1 = L / 2 + 1;
    return up256(sizeof(DevReplica) * R) + up256(sizeof(int) * R) +
           up256(sizeof(DevCounters) * R) + up256(H1 * H1 * 4) + up256(sizeof(int)) +
           refresh_tc_scratch_bytes(L * L, 2, R);
}

}  // namespace cg

extern "C" int cg_refresh_tc_noalloc(int L, int R, double nu, const unsigned int *occ,
                                     const double *phi, float *eps, double *max_err,
                                     void *stream)
{
    using namespace cg;
    if (L < 16 || L > 1024 || (L & 1) || (L * L) % 128 != 0) {
        set_last_error("cg_refresh_tc_noalloc: L must be even, 16 <= L <= 1024, L*L a "
                       "multiple of 128");
        return CG_EINVAL;
    }
    if (R < 1 || R > 512) {
        set_last_error("cg_refresh_tc_noalloc: R must be in [1, 512]");
        return CG_EINVAL;
    }
    if (!(nu > 0.0 && nu < 1.0)) {
        set_last_error("cg_refresh_tc_noalloc: nu must be in (0, 1)");
        return CG_EINVAL;
    }
    if (!occ || !phi || !eps) {
        set_last_error("cg_refresh_tc_noalloc: occ, phi and eps are required");
        return CG_EINVAL;
    }
    const size_t need = noalloc_scratch_bytes(L, R);
    if (need > kStaticScratchBytes) {
        set_last_error("cg_refresh_tc_noalloc: L=" + std::to_string(L) + ", R=" +
                       std::to_string(R) + " needs " + std::to_string(need) +
                       " bytes of scratch; the static maximum is " +
                       std::to_string(kStaticScratchBytes) + " bytes (32 MiB)");
        return CG_EINVAL;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return CG_ECUDA;
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc) return rc;

    // carve the static scratch
    const int H1 = L / 2 + 1;
    unsigned char *p = base;
    DevReplica *d_reps = reinterpret_cast<DevReplica *>(p);
    p += up256(sizeof(DevReplica) * R);
    int *d_index = reinterpret_cast<int *>(p);
    p += up256(sizeof(int) * R);
    DevCounters *d_ctr = reinterpret_cast<DevCounters *>(p);
    p += up256(sizeof(DevCounters) * R);
    uint32_t *d_tab = reinterpret_cast<uint32_t *>(p);
    p += up256((size_t)H1 * H1 * 4);
    int *d_err = reinterpret_cast<int *>(p);
    p += up256(sizeof(int));
    unsigned char *d_scratch = p;

    // sum_{t != s} 1/r_st on the L x L torus (rows dy outer, dx inner)
    double C0 = 0.0;
    for (int dy = 0; dy < L; ++dy)
        for (int dx = 0; dx < L; ++dx) {
            const int fy = fold_axis(dy, L), fx = fold_axis(dx, L);
            C0 += (fx == 0 && fy == 0) ? 0.0 : 1.0 / std::sqrt((double)(fx * fx + fy * fy));
        }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    static_setup_kernel<<<(R + 127) / 128, 128, 0, st>>>(d_reps, d_index, d_ctr, d_err, R, L, nu,
                                                         C0, occ, phi, eps);
    static_split_table_kernel<<<(H1 * H1 + 255) / 256, 256, 0, st>>>(d_tab, L);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_refresh_tc(d_reps, d_index, R, L, 2, d_tab, d_scratch, d_err, st);
    if (e == cudaSuccess && max_err) {
        static_err_out_kernel<<<(R + 127) / 128, 128, 0, st>>>(d_ctr, max_err, R);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_last_error(std::string("cg_refresh_tc_noalloc: ") + cudaGetErrorString(e));
        return CG_ECUDA;
    }
    int err = 0;
    e = cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_last_error(std::string("cg_refresh_tc_noalloc: ") + cudaGetErrorString(e));
        return CG_ECUDA;
    }
    if (err) {
        set_last_error("cg_refresh_tc_noalloc: a bounded wait of the contraction ran out");
        return CG_ETIMEOUT;
    }
    return CG_OK;
}
