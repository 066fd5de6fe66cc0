// Inlet density without any device allocation (lbm_inlet_density_noalloc).
//
// Some callers cannot let the library call cudaMalloc at the moment they need
// this value: processes whose device memory is fully reserved by another
// allocator (e.g. a framework's caching pool, where a second allocator would
// find no room), or real-time code that sizes all of its memory up front and
// must not stall in the allocator later.  For them, the inlet reduction below
// keeps its per-block partial sums and its ticket counter in a file-scope
// static device array of fixed size instead of in memory allocated per
// context or per call.
//
// The array belongs to the loaded library: every GPU that loads it holds
// kNoAllocScratchDoubles * 8 bytes until the process exits.  All calls share it
// and it keeps the last call's contents; the counter is cleared at every call.
// Calls whose kernels overlap on the GPU (different streams, or several host
// threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <utility>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kNoAllocBlock = 256;
// Partial sums for at most this many blocks: inlets of up to
// kNoAllocMaxBlocks * 256 = 524,288 pore nodes (e.g. a 724 x 724 plane).
constexpr int kNoAllocMaxBlocks = 2048;
// partials, then one slot for the ticket counter, padded to 256 bytes.
constexpr int kNoAllocScratchDoubles = kNoAllocMaxBlocks + 32;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol's name is only a host-side handle, never a device address, so it is
// looked up once per device (with that device current) and cached.  The cached
// address belongs to the device context that was current at the lookup: after
// a cudaDeviceReset on that device it is stale, and the entry point must not
// be called again in that process.
cudaError_t scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

template <int... Qs, class F>
__device__ __forceinline__ void for_each_q(std::integer_sequence<int, Qs...>, F&& f) {
    (f(std::integral_constant<int, Qs>{}), ...);
}

// Same arithmetic as the context's inlet reduction: K'_i in FP64 per inlet pore
// node, fixed-shape block sums, last block sums the partials in index order and
// writes rho_in = 1 + (Q + sum K'_i) / A  (Eq. potential, rho0 = 1).
template <class S>
__global__ void __launch_bounds__(kNoAllocBlock)
k_inlet_density_noalloc(const typename S::T* __restrict__ fin, DevLattice L, const BcState* bc,
                        double* __restrict__ scratch, double* __restrict__ rho_in_out) {
    __shared__ double sh[32];
    __shared__ bool last;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoAllocMaxBlocks);
    const int64_t i64 = (int64_t)blockIdx.x * kNoAllocBlock + threadIdx.x;
    double k = 0.0;
    if (i64 < L.a_in) {
        const int i = (int)i64;
        const int64_t p = L.vox[i];
        using M = typename S::M;
        M r_own = M(0), g = M(0);
        if constexpr (S::kRef) {
            r_own = ref_at<M>(bc, plane_of((uint64_t)p, L.sz_magic));
            g = ref_slope<M>(bc);
        }
        M d[19];
        for_each_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 6, 7, 8, 9, 10, 12, 13, 16, 17>{},
                   [&](auto qc) {
                       constexpr int Q = decltype(qc)::value;
                       d[Q] = pull<S, Q>(fin, L.ns, L.grid, p, i, L.sy, L.sz, r_own, g);
                   });
        k = (double)d[0] + (double)d[1] + (double)d[2] + (double)d[3] + (double)d[4] +
            (double)d[7] + (double)d[8] + (double)d[9] + (double)d[10] +
            2.0 * ((double)d[6] + (double)d[12] + (double)d[13] + (double)d[16] + (double)d[17]);
    }
    // block sum (warp shuffles, then the first warp)
    for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = k;
    __syncthreads();
    if (wid == 0) {
        double b = lane < kNoAllocBlock / 32 ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
        if (lane == 0) {
            scratch[blockIdx.x] = b;
            __threadfence();
            last = atomicAdd(counter, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += kNoAllocBlock) s += __ldcg(scratch + j);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (wid == 0) {
        double t = lane < kNoAllocBlock / 32 ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) {
            *rho_in_out = 1.0 + (bc->Q + t) / (double)L.a_in;
            *counter = 0u;
        }
    }
}

}  // namespace

int64_t noalloc_max_inlet_nodes() { return (int64_t)kNoAllocMaxBlocks * kNoAllocBlock; }

cudaError_t launch_inlet_density_noalloc(int prec, const void* fin, const DevLattice& L,
                                         const BcState* bc, double* rho_in_out, cudaStream_t st) {
    if (L.a_in < 1 || L.a_in > noalloc_max_inlet_nodes()) return cudaErrorInvalidValue;
    double* scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) return e;
    // the ticket counter must start at zero (a cleared 4-byte word; no allocation)
    e = cudaMemsetAsync(scratch + kNoAllocMaxBlocks, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((L.a_in + kNoAllocBlock - 1) / kNoAllocBlock);
    switch (prec) {
        case 0:
            k_inlet_density_noalloc<StoreF64><<<nb, kNoAllocBlock, 0, st>>>(
                (const double*)fin, L, bc, scratch, rho_in_out);
            break;
        case 1:
            k_inlet_density_noalloc<StoreF32><<<nb, kNoAllocBlock, 0, st>>>(
                (const float*)fin, L, bc, scratch, rho_in_out);
            break;
        case 2:
            k_inlet_density_noalloc<StoreF16><<<nb, kNoAllocBlock, 0, st>>>(
                (const __half*)fin, L, bc, scratch, rho_in_out);
            break;
        case 3:
            k_inlet_density_noalloc<StoreBF16><<<nb, kNoAllocBlock, 0, st>>>(
                (const __nv_bfloat16*)fin, L, bc, scratch, rho_in_out);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm
