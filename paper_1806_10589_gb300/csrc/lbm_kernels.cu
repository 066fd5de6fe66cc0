// CUDA kernels of the D3Q19 flux-boundary step (sm_103a).
//
//   k_inlet_reduce  Eq. (potential): inlet density from the pulled known sums of
//                   all inlet pore nodes, FP64 warp-shuffle/block reduction and
//                   a deterministic last-block finish.
//   k_step          one full time step for every pore node: pull streaming with
//                   halfway bounce-back (Eq. LBE), the Appendix B closures at the
//                   inlet/outlet planes, collision (Appendix A) and the store.
//   k_monitors      FP64 mass / flux / max|u| / NaN reductions of a state.
//   k_export, k_init_eq, k_encode, k_decode   field and state conversions.
#include <utility>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kBlock = 256;
constexpr int kReduceBlock = 256;

template <int... Qs, class F>
__device__ __forceinline__ void for_q(std::integer_sequence<int, Qs...>, F&& f) {
    (f(std::integral_constant<int, Qs>{}), ...);
}
using AllQ = std::make_integer_sequence<int, 19>;

template <class S>
__device__ __forceinline__ void pull_all(typename S::M* d, const typename S::T* __restrict__ fin,
                                         const DevLattice& L, int64_t p, int i) {
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[Q] = pull<S, Q>(fin, L.ns, L.grid, p, i, L.sy, L.sz);
    });
}

template <class S>
__device__ __forceinline__ void store_all(const typename S::M* d, typename S::T* __restrict__ fout,
                                          int64_t ns, int i) {
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        fout[(int64_t)Q * ns + i] = S::template enc<Q>(d[Q]);
    });
}

// ------------------------------------------------------------ reductions ---
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
// Fixed-shape block sum: the result depends only on the inputs, not on timing.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;  // valid in thread 0
}
template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
        r = warp_max(r);
    }
    __syncthreads();
    return r;
}

// ------------------------------------------------------- inlet reduction ---
// One thread per inlet pore node (pore indices [0, A)).  K'_i is the known sum
// of Eq. (inlet) on shifted values, formed in FP64; S' = sum_i K'_i; then
// rho_in - 1 = (Q + S') / A  (Eq. potential with rho0 = 1, since K = 1 + K').
template <class S>
__global__ void __launch_bounds__(kReduceBlock)
k_inlet_reduce(const typename S::T* __restrict__ fin, DevLattice L, BcState* bc,
               double* __restrict__ partials, unsigned* __restrict__ counter) {
    __shared__ double sh[32];
    __shared__ bool last;
    if (bc->inlet_mode != 0) {  // fixed-pressure inlet: nothing to reduce
        if (blockIdx.x == 0 && threadIdx.x == 0) bc->drho_in = bc->drho_in_fixed;
        return;
    }
    const int64_t i64 = (int64_t)blockIdx.x * kReduceBlock + threadIdx.x;
    double k = 0.0;
    if (i64 < L.a_in) {
        const int i = (int)i64;
        const int64_t p = L.vox[i];
        using M = typename S::M;
        M d[19];
        for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 6, 7, 8, 9, 10, 12, 13, 16, 17>{},
              [&](auto qc) {
                  constexpr int Q = decltype(qc)::value;
                  d[Q] = pull<S, Q>(fin, L.ns, L.grid, p, i, L.sy, L.sz);
              });
        k = (double)d[0] + (double)d[1] + (double)d[2] + (double)d[3] + (double)d[4] +
            (double)d[7] + (double)d[8] + (double)d[9] + (double)d[10] +
            2.0 * ((double)d[6] + (double)d[12] + (double)d[13] + (double)d[16] + (double)d[17]);
    }
    const double b = block_sum<kReduceBlock>(k, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += kReduceBlock) s += __ldcg(partials + j);
    s = block_sum<kReduceBlock>(s, sh);
    if (threadIdx.x == 0) {
        bc->drho_in = (bc->Q + s) / (double)L.a_in;
        *counter = 0u;
    }
}

// ---------------------------------------------------------- the step ---
template <class S>
__global__ void __launch_bounds__(kBlock)
k_step(const typename S::T* __restrict__ fin, typename S::T* __restrict__ fout, DevLattice L,
       typename S::M sp, typename S::M sm, const BcState* __restrict__ bc) {
    using M = typename S::M;
    const int64_t i64 = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (i64 >= L.n) return;
    const int i = (int)i64;
    const int64_t p = __ldg(L.vox + i);
    M d[19];
    pull_all<S>(d, fin, L, p, i);
    if (i < L.a_in) {
        // Section 2: after streaming, before collision.  u_z from Eq. (inlet)
        // with the density of Eq. (potential); then the Appendix B closure.
        const M uz = M(bc->drho_in) - inlet_known(d);
        close_inlet(d, uz);
    } else if (i64 >= L.n - L.a_out) {
        const M uz = outlet_known(d) - M(bc->drho_out);
        close_outlet(d, uz);
    }
    collide(d, sp, sm);
    store_all<S>(d, fout, L.ns, i);
}

// ---------------------------------------------------------- monitors ---
template <class S>
__global__ void __launch_bounds__(kReduceBlock)
k_monitors(const typename S::T* __restrict__ f, DevLattice L, double* __restrict__ partials,
           unsigned* __restrict__ counter, MonitorOut* out) {
    using M = typename S::M;
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i64 = (int64_t)blockIdx.x * kReduceBlock + threadIdx.x;
    double v[5] = {0, 0, 0, 0, 0};
    if (i64 < L.n) {
        const int i = (int)i64;
        M d[19];
        for_q(AllQ{}, [&](auto qc) {
            constexpr int Q = decltype(qc)::value;
            d[Q] = S::template dec<Q>(f[(int64_t)Q * L.ns + i]);
        });
        M drho, jx, jy, jz;
        moments(d, drho, jx, jy, jz);
        const double u2 = (double)jx * jx + (double)jy * jy + (double)jz * jz;
        const bool bad = !isfinite((double)drho) || !isfinite(u2);
        v[0] = bad ? 0.0 : (double)drho;
        if (i64 < L.a_in && !bad) v[1] = (double)jz;
        if (i64 >= L.n - L.a_out && !bad) v[2] = (double)jz;
        v[3] = bad ? 0.0 : u2;
        v[4] = bad ? 1.0 : 0.0;
    }
    const int nb = gridDim.x;
    double r[5];
    r[0] = block_sum<kReduceBlock>(v[0], sh);
    r[1] = block_sum<kReduceBlock>(v[1], sh);
    r[2] = block_sum<kReduceBlock>(v[2], sh);
    r[3] = block_max<kReduceBlock>(v[3], sh);
    r[4] = block_sum<kReduceBlock>(v[4], sh);
    if (threadIdx.x == 0) {
        for (int c = 0; c < 5; ++c) partials[(int64_t)c * nb + blockIdx.x] = r[c];
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[5] = {0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < nb; j += kReduceBlock) {
        acc[0] += __ldcg(partials + j);
        acc[1] += __ldcg(partials + (int64_t)nb + j);
        acc[2] += __ldcg(partials + 2 * (int64_t)nb + j);
        acc[3] = fmax(acc[3], __ldcg(partials + 3 * (int64_t)nb + j));
        acc[4] += __ldcg(partials + 4 * (int64_t)nb + j);
    }
    const double t0 = block_sum<kReduceBlock>(acc[0], sh);
    const double t1 = block_sum<kReduceBlock>(acc[1], sh);
    const double t2 = block_sum<kReduceBlock>(acc[2], sh);
    const double t3 = block_max<kReduceBlock>(acc[3], sh);
    const double t4 = block_sum<kReduceBlock>(acc[4], sh);
    if (threadIdx.x == 0) {
        out->drho_sum = t0;
        out->q_in = t1;
        out->q_out = t2;
        out->umax2 = t3;
        out->nan_count = t4;
        *counter = 0u;
    }
}

// ---------------------------------------------------- conversions ---
__device__ __forceinline__ int64_t unpadded(const DevLattice& L, int64_t p) {
    const int64_t z = p / L.sz - 1;
    const int64_t rem = p % L.sz;
    const int64_t y = rem / L.sy - 1;
    const int64_t x = rem % L.sy - 1;
    return (z * L.ny + y) * L.nx + x;
}

template <class S, class O>
__global__ void k_export(const typename S::T* __restrict__ f, DevLattice L, O* rho, O* ux, O* uy,
                         O* uz) {
    using M = typename S::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    M d[19];
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[Q] = S::template dec<Q>(f[(int64_t)Q * L.ns + i]);
    });
    M drho, jx, jy, jz;
    moments(d, drho, jx, jy, jz);
    const int64_t o = unpadded(L, L.vox[i]);
    if (rho) rho[o] = (O)(1.0 + (double)drho);
    if (ux) ux[o] = (O)jx;
    if (uy) uy[o] = (O)jy;
    if (uz) uz[o] = (O)jz;
}

template <class S>
__global__ void k_init_eq(typename S::T* __restrict__ f, DevLattice L, const double* rho,
                          const double* ux, const double* uy, const double* uz) {
    using M = typename S::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const M dr = rho ? M(rho[i] - 1.0) : M(0);
    const M u[3] = {ux ? M(ux[i]) : M(0), uy ? M(uy[i]) : M(0), uz ? M(uz[i]) : M(0)};
    const M uu15 = M(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        const M xu = M(cx(Q)) * u[0] + M(cy(Q)) * u[1] + M(cz(Q)) * u[2];
        const M dq = M(wq(Q)) * (dr + M(3) * xu + M(4.5) * xu * xu - uu15);
        f[(int64_t)Q * L.ns + i] = S::template enc<Q>(dq);
    });
}

template <class S>
__global__ void k_encode(typename S::T* __restrict__ f, DevLattice L, const double* __restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        f[(int64_t)Q * L.ns + i] = S::template enc<Q>((typename S::M)d[(int64_t)Q * L.n + i]);
    });
}

template <class S>
__global__ void k_decode(const typename S::T* __restrict__ f, DevLattice L, double* __restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[(int64_t)Q * L.n + i] = (double)S::template dec<Q>(f[(int64_t)Q * L.ns + i]);
    });
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class F>
cudaError_t dispatch(int prec, F&& f) {
    switch (prec) {
        case 0: return f(StoreF64{});
        case 1: return f(StoreF32{});
        case 2: return f(StoreF16{});
        case 3: return f(StoreBF16{});
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int elem_size(int prec) { return prec == 0 ? 8 : prec == 1 ? 4 : 2; }
int inlet_reduce_blocks(const DevLattice& L) { return (int)blocks_for(L.a_in, kReduceBlock); }
int monitor_blocks(const DevLattice& L) { return (int)blocks_for(L.n, kReduceBlock); }

cudaError_t launch_inlet_reduce(int prec, const void* fin, const DevLattice& L, BcState* bc,
                                double* partials, unsigned* counter, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_inlet_reduce<S><<<inlet_reduce_blocks(L), kReduceBlock, 0, st>>>(
            (const typename S::T*)fin, L, bc, partials, counter);
        return cudaGetLastError();
    });
}

cudaError_t launch_step(int prec, const void* fin, void* fout, const DevLattice& L, Relax r,
                        const BcState* bc, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        using M = typename S::M;
        k_step<S><<<blocks_for(L.n, kBlock), kBlock, 0, st>>>(
            (const typename S::T*)fin, (typename S::T*)fout, L, (M)r.sp, (M)r.sm, bc);
        return cudaGetLastError();
    });
}

cudaError_t launch_monitors(int prec, const void* f, const DevLattice& L, double* partials,
                            unsigned* counter, MonitorOut* out, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_monitors<S><<<monitor_blocks(L), kReduceBlock, 0, st>>>((const typename S::T*)f, L,
                                                                   partials, counter, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_export(int prec, const void* f, const DevLattice& L, void* rho, void* ux,
                          void* uy, void* uz, int out_double, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        if (out_double)
            k_export<S, double><<<blocks_for(L.n, 256), 256, 0, st>>>(
                (const typename S::T*)f, L, (double*)rho, (double*)ux, (double*)uy, (double*)uz);
        else
            k_export<S, float><<<blocks_for(L.n, 256), 256, 0, st>>>(
                (const typename S::T*)f, L, (float*)rho, (float*)ux, (float*)uy, (float*)uz);
        return cudaGetLastError();
    });
}

cudaError_t launch_init_eq(int prec, void* f, const DevLattice& L, const double* rho,
                           const double* ux, const double* uy, const double* uz, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_init_eq<S><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L, rho, ux, uy, uz);
        return cudaGetLastError();
    });
}

cudaError_t launch_encode(int prec, void* f, const DevLattice& L, const double* d, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_encode<S><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L, d);
        return cudaGetLastError();
    });
}

cudaError_t launch_decode(int prec, const void* f, const DevLattice& L, double* d, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_decode<S><<<blocks_for(L.n, 256), 256, 0, st>>>((const typename S::T*)f, L, d);
        return cudaGetLastError();
    });
}

}  // namespace lbm
