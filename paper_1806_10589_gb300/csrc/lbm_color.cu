// Two-fluid colour model (Appendix A) on the same lattice, with the paper's
// flux inlet and pressure outlet, FP64 or FP32 storage (arithmetic in the
// storage type).  Per step:
//   k_color_pre   phase field phi = (N_A - N_B)/(N_A + N_B) of every pore node
//                 (D3Q7 sums), and the inlet density of Eq. (potential) from the
//                 pulled momentum distributions (FP64 sum, last-block finish);
//   k_color_step  pull of the 19 momentum distributions with halfway bounce-back,
//                 Appendix B closures, colour gradient C = 3 sum_q w_q xi_q phi(x+xi_q)
//                 (solid voxels give phi_s, neighbours outside the box the node's
//                 own phi: the box faces are wetting-neutral), MRT collision with the interfacial equilibrium terms, then
//                 the D3Q7 mass transport: every node pushes
//                 A_q = w_q N_A [1 + 9/2 u.xi_q + beta N_B n.xi_q] (and B with -beta N_A)
//                 to x + xi_q, bouncing back from solids and lateral box faces; the outlet takes
//                 w6 N (1 - 9/2 u_z).  The inlet plane holds the injected
//                 composition: the pre-pass sets the value that entered each inlet
//                 node through the inlet so the node carries rho0 (1 +- phi_in)/2,
//                 rho0 = 1.
// Momentum distributions are stored shifted (d = f - w) as in the single-fluid
// path; A and B are stored as they are.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kCB = 256;
// Lateral out-of-box cell of the colour grid: a wall for momentum and mass
// transport (bounce-back) but wetting-neutral in the colour gradient.
constexpr int kSideOut = -3;

struct ColorParams {
    double Q;         // prescribed inlet flux
    double drho_out;  // outlet density - 1
    double drho_in;   // inlet density - 1 of the current step (output of k_color_pre)
    double phi_in;    // phase of the injected fluid
};

// Identity codec over the storage type (pull<> helper interface).
template <class T_>
struct StoreIdent {
    using T = T_;
    using M = T_;
    template <int Q> __device__ static M dec(T v, M) { return v; }
    template <int Q> __device__ static T enc(M v, M) { return v; }
};

template <int... Qs, class F>
__device__ __forceinline__ void for_q(std::integer_sequence<int, Qs...>, F&& f) {
    (f(std::integral_constant<int, Qs>{}), ...);
}
using AllQ = std::make_integer_sequence<int, 19>;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < kCB / 32 ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// D3Q7 weights (Appendix A): w0 = 1/3, w1..6 = 1/9.
__host__ __device__ constexpr double w7(int q) { return q == 0 ? 1.0 / 3.0 : 1.0 / 9.0; }

// Rows of the d'Humieres moment matrix that carry the interfacial terms and
// their squared norms (the matrix is orthogonal, so its inverse is the
// transpose scaled by 1 / norm^2).
__host__ __device__ constexpr double mrow(int k, int q) {
    return k == 1 ? 19.0 * (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) - 30.0
         : k == 9 ? 3.0 * cx(q) * cx(q) - (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q))
         : k == 11 ? double(cy(q) * cy(q) - cz(q) * cz(q))
         : k == 13 ? double(cx(q) * cy(q))
         : k == 14 ? double(cy(q) * cz(q))
         : double(cx(q) * cz(q));
}
__host__ __device__ constexpr double mnorm2(int k) {
    double s = 0.0;
    for (int q = 0; q < 19; ++q) s += mrow(k, q) * mrow(k, q);
    return s;
}

template <class T>
__global__ void __launch_bounds__(kCB)
k_color_pre(const T* __restrict__ f, T* __restrict__ A, T* __restrict__ B, T* __restrict__ phi,
            DevLattice L, ColorParams* prm, double* __restrict__ partials, unsigned* __restrict__ counter) {
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i64 = (int64_t)blockIdx.x * kCB + threadIdx.x;
    double k = 0.0;
    if (i64 < L.n) {
        const int i = (int)i64;
        T na = 0, nb = 0;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            if (q == 5 && i64 < L.a_in) continue;
            na += A[(int64_t)q * L.ns + i];
            nb += B[(int64_t)q * L.ns + i];
        }
        if (i64 < L.a_in) {
            // injected composition at the reference density rho0 = 1 (the momentum
            // density carries the pressure, the phase densities do not)
            const T fa = (T(1) + T(prm->phi_in)) * T(0.5);
            A[(int64_t)5 * L.ns + i] = fa - na;
            B[(int64_t)5 * L.ns + i] = (T(1) - fa) - nb;
            na = fa;
            nb = T(1) - fa;
        }
        phi[i] = (na - nb) / (na + nb);
        if (i64 < L.a_in) {
            const int64_t p = L.vox[i];
            T d[19];
            for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 6, 7, 8, 9, 10, 12, 13, 16, 17>{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value;
                d[Q] = pull<StoreIdent<T>, Q>(f, L.ns, L.grid, p, i, L.sy, L.sz, T(0), T(0));
            });
            k = (double)d[0] + (double)d[1] + (double)d[2] + (double)d[3] + (double)d[4] + (double)d[7] +
                (double)d[8] + (double)d[9] + (double)d[10] +
                2.0 * ((double)d[6] + (double)d[12] + (double)d[13] + (double)d[16] + (double)d[17]);
        }
    }
    if (L.a_in > 0 && (int64_t)blockIdx.x * kCB < L.a_in) {  // block-uniform
        const unsigned nbk = (unsigned)((L.a_in + kCB - 1) / kCB);
        const double b = block_sum(k, sh);
        if (threadIdx.x == 0) {
            partials[blockIdx.x] = b;
            __threadfence();
            last = atomicAdd(counter, 1u) == nbk - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            double s = 0.0;
            for (unsigned j = threadIdx.x; j < nbk; j += kCB) s += __ldcg(partials + j);
            s = block_sum(s, sh);
            if (threadIdx.x == 0) {
                prm->drho_in = (prm->Q + s) / (double)L.a_in;
                *counter = 0u;
            }
        }
    }
}

// Row pointers of the two momentum buffers and the D3Q7 buffers of this step, as
// kernel parameters (constant bank): no registers spent on row addresses.
template <class T>
struct ColorRows {
    const T* fin[19];
    T* fout[19];
    const T* ain[7];
    T* aout[7];
    const T* bin[7];
    T* bout[7];
};

#ifndef LBM_COLOR_MIN_BLOCKS
#define LBM_COLOR_MIN_BLOCKS 4
#endif
// LBM_COLOR_PREFETCH: the step asks L2 for the rows of the block that many
// blocks ahead (bulk prefetch, nothing waited for); 0 = off.  Measured on the
// 192x192x384 pack: 32 best (-5.6 % per step), 256 slower than none.
#ifndef LBM_COLOR_PREFETCH
#define LBM_COLOR_PREFETCH 32
#endif
template <class T>
constexpr int color_min_blocks() {
    return sizeof(T) == 8 ? 1 : LBM_COLOR_MIN_BLOCKS;
}

// OFF32 (buffers of 19 ns < 2^32 elements): a gathered momentum value and a
// pushed D3Q7 value are addressed as row 0 plus one 32-bit element offset, the
// row chosen by a 32-bit select (as in the single-fluid gather-scatter step).
template <class T, bool OFF32 = false>
__global__ void __launch_bounds__(kCB, color_min_blocks<T>())
k_color_step(const ColorRows<T> R, const T* __restrict__ phi, DevLattice L, const ColorParams* __restrict__ prm,
             T sp, T sm, T alpha, T beta, T phi_s) {
    const int64_t i64 = (int64_t)blockIdx.x * kCB + threadIdx.x;
    if constexpr (LBM_COLOR_PREFETCH > 0) {
        // threads 0..18: momentum rows, 19..25: A rows, 26..32: B rows (rows of ns
        // elements from row 0, as launched), 33: phi, 34: the voxel list cut to a
        // multiple of 4 entries
        const int64_t s = ((int64_t)blockIdx.x + LBM_COLOR_PREFETCH) * kCB;
        const int t = (int)threadIdx.x;
        if (t < 19) l2_prefetch_range(R.fin[0] + (int64_t)t * L.ns, s, kCB, L.ns);
        else if (t < 26) l2_prefetch_range(R.ain[0] + (int64_t)(t - 19) * L.ns, s, kCB, L.ns);
        else if (t < 33) l2_prefetch_range(R.bin[0] + (int64_t)(t - 26) * L.ns, s, kCB, L.ns);
        else if (t == 33) l2_prefetch_range(phi, s, kCB, L.ns);
        else if (t == 34) l2_prefetch_range(L.vox, s, kCB, L.n & ~(int64_t)3);
    }
    if (i64 >= L.n) return;
    const int i = (int)i64;
    const uint64_t pol = l2_policy_evict_last();  // index structures stay in L2
    const uint32_t p = ld_hint(reinterpret_cast<const unsigned*>(L.vox) + i, pol);
    const T phi_own = phi[i];
    T d[19];
    T cgx = 0, cgy = 0, cgz = 0;
    d[0] = R.fin[0][i];
    for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value + 1;
        const int id = ld_hint(L.grid + (uint32_t)(p + (uint32_t)grid_off<Q>(L.sy, L.sz)), pol);
        if constexpr (OFF32)
            d[Q] = R.fin[0][id >= 0 ? (uint32_t)Q * (uint32_t)L.ns + (uint32_t)id
                                    : (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)i];
        else
            d[Q] = id >= 0 ? R.fin[Q][id] : R.fin[opp(Q)][i];
        // colour-gradient neighbour x + xi_opp(Q) is the pull source of Q
        const T ph = id >= 0 ? phi[id] : (id == SOLID ? phi_s : phi_own);  // box faces: own phi
        constexpr int Rq = opp(Q);  // this neighbour sits at x + xi_Rq
        const T wq3 = T(3.0 * wq(Rq));
        if (cx(Rq)) cgx += wq3 * T(cx(Rq)) * ph;
        if (cy(Rq)) cgy += wq3 * T(cy(Rq)) * ph;
        if (cz(Rq)) cgz += wq3 * T(cz(Rq)) * ph;
    });
    if (i < L.a_in) {
        close_inlet(d, T(prm->drho_in) - inlet_known(d));
    } else if (i64 >= L.n - L.a_out) {
        close_outlet(d, outlet_known(d) - T(prm->drho_out));
    }
    T drho, jx, jy, jz;
    moments(d, drho, jx, jy, jz);
    // interfacial equilibrium terms (relaxed at s_nu, like every even moment they enter)
    const T cmag = sqrt(cgx * cgx + cgy * cgy + cgz * cgz);
    const T inv = cmag > T(0) ? T(1) / cmag : T(0);
    const T nx = cgx * inv, ny = cgy * inv, nz = cgz * inv;
    const T a = alpha * cmag;
    const T dm1 = a, dm9 = T(0.5) * a * (T(2) * nx * nx - ny * ny - nz * nz), dm11 = T(0.5) * a * (ny * ny - nz * nz);
    const T dm13 = T(0.5) * a * nx * ny, dm14 = T(0.5) * a * ny * nz, dm15 = T(0.5) * a * nx * nz;
    collide(d, sp, sm);
    // an opaque copy of i for the stores (sharing the load addresses would keep
    // them live across the collision)
    int j;
    asm volatile("mov.b32 %0, %1;" : "=r"(j) : "r"(i));
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        const T df = T(mrow(1, Q) / mnorm2(1)) * dm1 + T(mrow(9, Q) / mnorm2(9)) * dm9 +
                     T(mrow(11, Q) / mnorm2(11)) * dm11 + T(mrow(13, Q) / mnorm2(13)) * dm13 +
                     T(mrow(14, Q) / mnorm2(14)) * dm14 + T(mrow(15, Q) / mnorm2(15)) * dm15;
        R.fout[Q][j] = d[Q] + sp * df;
    });
    // D3Q7 mass transport with recolouring (push); destinations looked up again
    T na = 0, nb = 0;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        na += R.ain[q][j];
        nb += R.bin[q][j];
    }
    const bool inlet = j < L.a_in, outlet = (int64_t)j >= L.n - L.a_out;
    const uint32_t ps = ld_hint(reinterpret_cast<const unsigned*>(L.vox) + j, pol);
    for_q(std::make_integer_sequence<int, 7>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        const T xu = T(cx(Q)) * jx + T(cy(Q)) * jy + T(cz(Q)) * jz;
        const T xn = T(cx(Q)) * nx + T(cy(Q)) * ny + T(cz(Q)) * nz;
        const T va = T(w7(Q)) * na * (T(1) + T(4.5) * xu + beta * nb * xn);
        const T vb = T(w7(Q)) * nb * (T(1) + T(4.5) * xu - beta * na * xn);
        if constexpr (Q == 0) {
            R.aout[0][j] = va;
            R.bout[0][j] = vb;
        } else {
            // push destination x + xi_Q is the pull source of opp(Q)
            const int id = ld_hint(L.grid + (uint32_t)(ps + (uint32_t)grid_off<opp(Q)>(L.sy, L.sz)), pol);
            if constexpr (OFF32) {
                if (id != ZOUT) {  // a pore, or bounce-back from a solid voxel or lateral box face
                    const uint32_t off = id >= 0 ? (uint32_t)Q * (uint32_t)L.ns + (uint32_t)id
                                                 : (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)j;
                    R.aout[0][off] = va;
                    R.bout[0][off] = vb;
                }
            } else if (id >= 0) {
                R.aout[Q][id] = va;
                R.bout[Q][id] = vb;
            } else if (id != ZOUT) {  // solid voxel or lateral box face: bounce back
                R.aout[opp(Q)][j] = va;
                R.bout[opp(Q)][j] = vb;
            }
        }
    });
    if (inlet) {  // the value entering through the inlet plane: set by the next pre-pass
        R.aout[5][j] = T(0);
        R.bout[5][j] = T(0);
    }
    if (outlet) {  // the value entering through the outlet plane (direction 6)
        R.aout[6][j] = T(w7(6)) * na * (T(1) - T(4.5) * jz);
        R.bout[6][j] = T(w7(6)) * nb * (T(1) - T(4.5) * jz);
    }
}

template <class T>
__global__ void k_color_export(const T* __restrict__ f, const T* __restrict__ phi, DevLattice L,
                               const int64_t* __restrict__ voxel, double* rho, double* ux, double* uy, double* uz,
                               double* ph) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    T d[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) d[q] = f[(int64_t)q * L.ns + i];
    T drho, jx, jy, jz;
    moments(d, drho, jx, jy, jz);
    const int64_t o = voxel[i];
    rho[o] = 1.0 + (double)drho;
    ux[o] = (double)jx;
    uy[o] = (double)jy;
    uz[o] = (double)jz;
    ph[o] = (double)phi[i];
}

template <class T>
__global__ void k_color_face_flux(const T* __restrict__ f, DevLattice L, int which, double* __restrict__ partials,
                                  unsigned* __restrict__ counter, double* out) {
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i = (int64_t)blockIdx.x * kCB + threadIdx.x;
    double v = 0.0;
    const bool on = i < L.n && (which == 0 ? i < L.a_in : i >= L.n - L.a_out);
    if (on) {
        T d[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) d[q] = f[(int64_t)q * L.ns + i];
        T drho, jx, jy, jz;
        moments(d, drho, jx, jy, jz);
        v = (double)jz;
    }
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned j = threadIdx.x; j < gridDim.x; j += kCB) s += __ldcg(partials + j);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        *out = s;
        *counter = 0u;
    }
}

// Rest state with a phase field: f = f^eq(rho, 0), A = w7 rho (1 + phi)/2,
// B = w7 rho (1 - phi)/2 (pore order inputs).
template <class T>
__global__ void k_color_init(T* __restrict__ f, T* __restrict__ A, T* __restrict__ B, DevLattice L,
                             const double* __restrict__ phi, const double* __restrict__ rho) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const double r = rho ? rho[i] : 1.0;
    const double ph = phi[i];
    for (int q = 0; q < 19; ++q) f[(int64_t)q * L.ns + i] = (T)(wq(q) * (r - 1.0));
    for (int q = 0; q < 7; ++q) {
        A[(int64_t)q * L.ns + i] = (T)(w7(q) * r * (1.0 + ph) * 0.5);
        B[(int64_t)q * L.ns + i] = (T)(w7(q) * r * (1.0 - ph) * 0.5);
    }
}

thread_local std::string g_color_err;

}  // namespace
}  // namespace lbm

struct lbm_color {
    int device = 0;
    int prec = 1;
    int nx = 0, ny = 0, nz = 0;
    double sp = 1, sm = 1, alpha = 0, beta = 0.95, phi_s = -1;
    lbm::DevLattice L{};
    void* f[2] = {nullptr, nullptr};
    void* A[2] = {nullptr, nullptr};
    void* B[2] = {nullptr, nullptr};
    void* phi = nullptr;
    int cur = 0;
    uint32_t* d_vox = nullptr;
    int* d_grid = nullptr;
    int64_t* d_voxel = nullptr;  // unpadded voxel of each pore node
    lbm::ColorParams h_prm{};
    lbm::ColorParams* d_prm = nullptr;
    double* d_partials = nullptr;
    unsigned* d_counter = nullptr;
    unsigned* d_counter2 = nullptr;
    double* d_out = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<int64_t> pore_voxel;
    int64_t steps = 0;
    int status = LBM_OK;
    std::string err;
};

namespace {

int cfail(lbm_color* c, int code, const char* fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = b;
        if (code == LBM_ECUDA) c->status = LBM_ECUDA;
    } else {
        lbm::g_color_err = b;
    }
    return code;
}
#define COLOR_CUDA(c, call)                                                                \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return cfail((c), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int center(lbm_color* c) {
    if (!c) return LBM_EINVAL;
    if (c->status == LBM_ECUDA) return LBM_ECUDA;
    COLOR_CUDA(c, cudaSetDevice(c->device));
    return LBM_OK;
}

void crelease(lbm_color* c) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->f[k]);
        cudaFree(c->A[k]);
        cudaFree(c->B[k]);
    }
    cudaFree(c->phi);
    cudaFree(c->d_vox);
    cudaFree(c->d_grid);
    cudaFree(c->d_voxel);
    cudaFree(c->d_prm);
    cudaFree(c->d_partials);
    cudaFree(c->d_counter);
    cudaFree(c->d_counter2);
    cudaFree(c->d_out);
}

template <class F>
cudaError_t cdispatch(int prec, F&& f) {
    if (prec == LBM_PREC_FP64) return f(double{});
    if (prec == LBM_PREC_FP32) return f(float{});
    return cudaErrorInvalidValue;
}

int cpush(lbm_color* c) {
    COLOR_CUDA(c, cudaMemcpyAsync(c->d_prm, &c->h_prm, sizeof(lbm::ColorParams), cudaMemcpyHostToDevice, c->stream));
    COLOR_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int cstep_once(lbm_color* c) {
    const unsigned nb = (unsigned)((c->L.n + lbm::kCB - 1) / lbm::kCB);
    const int k = c->cur;
    cudaError_t e = cdispatch(c->prec, [&](auto zero) {
        using T = decltype(zero);
        lbm::k_color_pre<T><<<nb, lbm::kCB, 0, c->stream>>>((const T*)c->f[k], (T*)c->A[k], (T*)c->B[k],
                                                           (T*)c->phi, c->L, c->d_prm, c->d_partials, c->d_counter);
        lbm::ColorRows<T> R;
        for (int q = 0; q < 19; ++q) {
            R.fin[q] = (const T*)c->f[k] + (int64_t)q * c->L.ns;
            R.fout[q] = (T*)c->f[k ^ 1] + (int64_t)q * c->L.ns;
        }
        for (int q = 0; q < 7; ++q) {
            R.ain[q] = (const T*)c->A[k] + (int64_t)q * c->L.ns;
            R.aout[q] = (T*)c->A[k ^ 1] + (int64_t)q * c->L.ns;
            R.bin[q] = (const T*)c->B[k] + (int64_t)q * c->L.ns;
            R.bout[q] = (T*)c->B[k ^ 1] + (int64_t)q * c->L.ns;
        }
        if (19 * (uint64_t)c->L.ns <= 0xFFFFFFFFull && !std::getenv("GB300_LBM_COLOR_ADDR64"))
            lbm::k_color_step<T, true><<<nb, lbm::kCB, 0, c->stream>>>(
                R, (const T*)c->phi, c->L, c->d_prm, (T)c->sp, (T)c->sm, (T)c->alpha, (T)c->beta, (T)c->phi_s);
        else
            lbm::k_color_step<T><<<nb, lbm::kCB, 0, c->stream>>>(R, (const T*)c->phi, c->L, c->d_prm, (T)c->sp,
                                                                 (T)c->sm, (T)c->alpha, (T)c->beta, (T)c->phi_s);
        return cudaGetLastError();
    });
    COLOR_CUDA(c, e);
    c->cur ^= 1;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_color_create(const uint8_t* mask, int nx, int ny, int nz, double tau, double alpha, double beta,
                     double phi_s, int precision, lbm_color** out) {
    lbm::g_color_err.clear();
    if (!out || !mask) return cfail(nullptr, LBM_EINVAL, "NULL argument");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nx > 2047 || ny > 2047 || nz < 3 || nz > 1023)
        return cfail(nullptr, LBM_EINVAL, "box %dx%dx%d out of range", nx, ny, nz);
    if (!(tau > 0.5) || !(tau < 1e6)) return cfail(nullptr, LBM_EINVAL, "tau must exceed 0.5");
    if (precision != LBM_PREC_FP64 && precision != LBM_PREC_FP32)
        return cfail(nullptr, LBM_EUNSUPPORTED, "the colour model stores FP64 or FP32");
    if (!(alpha >= 0) || !(beta >= 0) || !(beta <= 1) || !(phi_s >= -1) || !(phi_s <= 1))
        return cfail(nullptr, LBM_EINVAL, "need alpha >= 0, 0 <= beta <= 1, -1 <= phi_s <= 1");
    const int64_t px = nx + 2, py = ny + 2, pz = nz + 2;
    if (px * py * pz > (int64_t)UINT32_MAX) return cfail(nullptr, LBM_EINVAL, "box too large");
    auto* c = new (std::nothrow) lbm_color();
    if (!c) return cfail(nullptr, LBM_ENOMEM, "host allocation");
    cudaGetDevice(&c->device);
    c->prec = precision;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->sp = 1.0 / tau;
    c->sm = 8.0 * (2.0 - c->sp) / (8.0 - c->sp);
    c->alpha = alpha;
    c->beta = beta;
    c->phi_s = phi_s;
    std::vector<int> grid((size_t)(px * py * pz), lbm::SOLID);
    for (int64_t z = 0; z < pz; ++z)
        for (int64_t y = 0; y < py; ++y)
            for (int64_t x = 0; x < px; ++x)
                if (z == 0 || z == pz - 1)
                    grid[(size_t)((z * py + y) * px + x)] = lbm::ZOUT;
                else if (x == 0 || x == px - 1 || y == 0 || y == py - 1)
                    grid[(size_t)((z * py + y) * px + x)] = lbm::kSideOut;
    std::vector<uint32_t> vox;
    int64_t a_in = 0, a_out = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = (z * ny + y) * nx + x;
                if (mask[v] > 1) {
                    delete c;
                    return cfail(nullptr, LBM_EINVAL, "mask values must be 0 or 1");
                }
                if (mask[v]) continue;
                const int64_t p = ((z + 1) * py + (y + 1)) * px + (x + 1);
                grid[(size_t)p] = (int)vox.size();
                vox.push_back((uint32_t)p);
                c->pore_voxel.push_back(v);
                if (z == 0) ++a_in;
                if (z == nz - 1) ++a_out;
            }
    const int64_t n = (int64_t)vox.size();
    if (n == 0) {
        delete c;
        return cfail(nullptr, LBM_EINVAL, "no pore nodes");
    }
    c->L.n = n;
    c->L.ns = (n + 127) / 128 * 128;
    c->L.a_in = a_in;
    c->L.a_out = a_out;
    c->L.nx = nx;
    c->L.ny = ny;
    c->L.nz = nz;
    c->L.sy = (int)px;
    c->L.sz = (int)(px * py);
    const int es = precision == LBM_PREC_FP64 ? 8 : 4;
    const size_t fb = (size_t)19 * c->L.ns * es, ab = (size_t)7 * c->L.ns * es;
    cudaError_t e = cudaSuccess;
    auto Al = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
    };
    for (int k = 0; k < 2; ++k) {
        Al(&c->f[k], fb);
        Al(&c->A[k], ab);
        Al(&c->B[k], ab);
    }
    Al(&c->phi, (size_t)c->L.ns * es);
    Al(&c->d_vox, vox.size() * 4);
    Al(&c->d_grid, grid.size() * 4);
    Al(&c->d_voxel, c->pore_voxel.size() * 8);
    Al(&c->d_prm, sizeof(lbm::ColorParams));
    Al(&c->d_partials, (size_t)((n + lbm::kCB - 1) / lbm::kCB + 1) * sizeof(double));
    Al(&c->d_counter, sizeof(unsigned));
    Al(&c->d_counter2, sizeof(unsigned));
    Al(&c->d_out, sizeof(double));
    c->L.vox = c->d_vox;
    c->L.grid = c->d_grid;
    c->h_prm = lbm::ColorParams{0.0, 0.0, 0.0, 1.0};
    if (e == cudaSuccess) e = cudaMemcpy(c->d_vox, vox.data(), vox.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_grid, grid.data(), grid.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_voxel, c->pore_voxel.data(), c->pore_voxel.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_prm, &c->h_prm, sizeof c->h_prm, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_counter2, 0, sizeof(unsigned));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemset(c->f[k], 0, fb);
        if (e == cudaSuccess) e = cudaMemset(c->A[k], 0, ab);
        if (e == cudaSuccess) e = cudaMemset(c->B[k], 0, ab);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "lbm_color_create: %s",
              cudaGetErrorString(e));
        cudaGetLastError();
        crelease(c);
        delete c;
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
    *out = c;
    return LBM_OK;
}

int lbm_color_set_stream(lbm_color* c, void* s) {
    int rc = center(c);
    if (rc) return rc;
    c->stream = (cudaStream_t)s;
    return LBM_OK;
}

int lbm_color_set_flux_bc(lbm_color* c, double Q, double phi_in) {
    int rc = center(c);
    if (rc) return rc;
    if (c->L.a_in == 0) return cfail(c, LBM_EUNSUPPORTED, "the inlet plane has no pore nodes");
    if (!(Q == Q) || !(phi_in >= -1) || !(phi_in <= 1)) return cfail(c, LBM_EINVAL, "bad Q or phi_in");
    c->h_prm.Q = Q;
    c->h_prm.phi_in = phi_in;
    return cpush(c);
}

int lbm_color_set_state(lbm_color* c, const double* f, const double* A, const double* B) {
    int rc = center(c);
    if (rc) return rc;
    if (!f || !A || !B) return cfail(c, LBM_EINVAL, "NULL state");
    const int64_t n = c->L.n, ns = c->L.ns;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    const int es = c->prec == LBM_PREC_FP64 ? 8 : 4;
    std::vector<double> hf((size_t)(19 * ns), 0.0), ha((size_t)(7 * ns), 0.0), hb((size_t)(7 * ns), 0.0);
    for (int q = 0; q < 19; ++q)
        for (int64_t i = 0; i < n; ++i)
            hf[(size_t)(q * ns + i)] = f[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]] - lbm::wq(q);
    for (int q = 0; q < 7; ++q)
        for (int64_t i = 0; i < n; ++i) {
            ha[(size_t)(q * ns + i)] = A[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]];
            hb[(size_t)(q * ns + i)] = B[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]];
        }
    auto up = [&](void* dst, const std::vector<double>& h) -> cudaError_t {
        if (es == 8) return cudaMemcpy(dst, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
        std::vector<float> t(h.begin(), h.end());
        return cudaMemcpy(dst, t.data(), t.size() * 4, cudaMemcpyHostToDevice);
    };
    COLOR_CUDA(c, cudaStreamSynchronize(c->stream));
    COLOR_CUDA(c, up(c->f[c->cur], hf));
    COLOR_CUDA(c, up(c->A[c->cur], ha));
    COLOR_CUDA(c, up(c->B[c->cur], hb));
    c->steps = 0;
    return LBM_OK;
}

int lbm_color_set_phase(lbm_color* c, const double* phi, const double* rho) {
    int rc = center(c);
    if (rc) return rc;
    if (!phi) return cfail(c, LBM_EINVAL, "NULL phi");
    const int64_t n = c->L.n;
    std::vector<double> h((size_t)(2 * n), 1.0);
    for (int64_t i = 0; i < n; ++i) {
        const double v = phi[(size_t)c->pore_voxel[(size_t)i]];
        if (!(v >= -1.0) || !(v <= 1.0)) return cfail(c, LBM_EINVAL, "phi must lie in [-1, 1]");
        h[(size_t)i] = v;
        if (rho) h[(size_t)(n + i)] = rho[(size_t)c->pore_voxel[(size_t)i]];
    }
    double* d = nullptr;
    COLOR_CUDA(c, cudaMalloc(&d, h.size() * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cdispatch(c->prec, [&](auto zero) {
            using T = decltype(zero);
            lbm::k_color_init<T><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                (T*)c->f[c->cur], (T*)c->A[c->cur], (T*)c->B[c->cur], c->L, d, d + n);
            return cudaGetLastError();
        });
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cfail(c, LBM_ECUDA, "lbm_color_set_phase: %s", cudaGetErrorString(e));
    c->steps = 0;
    return LBM_OK;
}

int lbm_color_get_state(lbm_color* c, double* f, double* A, double* B) {
    int rc = center(c);
    if (rc) return rc;
    const int64_t n = c->L.n, ns = c->L.ns;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    const int es = c->prec == LBM_PREC_FP64 ? 8 : 4;
    auto down = [&](const void* src, size_t cnt, std::vector<double>& h) -> cudaError_t {
        h.resize(cnt);
        if (es == 8) return cudaMemcpy(h.data(), src, cnt * 8, cudaMemcpyDeviceToHost);
        std::vector<float> t(cnt);
        cudaError_t e = cudaMemcpy(t.data(), src, cnt * 4, cudaMemcpyDeviceToHost);
        for (size_t k = 0; k < cnt; ++k) h[k] = t[k];
        return e;
    };
    COLOR_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<double> hf, ha, hb;
    COLOR_CUDA(c, down(c->f[c->cur], (size_t)(19 * ns), hf));
    COLOR_CUDA(c, down(c->A[c->cur], (size_t)(7 * ns), ha));
    COLOR_CUDA(c, down(c->B[c->cur], (size_t)(7 * ns), hb));
    if (f) {
        std::memset(f, 0, 19 * ncell * sizeof(double));
        for (int q = 0; q < 19; ++q)
            for (int64_t i = 0; i < n; ++i)
                f[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]] = lbm::wq(q) + hf[(size_t)(q * ns + i)];
    }
    for (int pass = 0; pass < 2; ++pass) {
        double* dst = pass ? B : A;
        const std::vector<double>& src = pass ? hb : ha;
        if (!dst) continue;
        std::memset(dst, 0, 7 * ncell * sizeof(double));
        for (int q = 0; q < 7; ++q)
            for (int64_t i = 0; i < n; ++i)
                dst[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]] = src[(size_t)(q * ns + i)];
    }
    return LBM_OK;
}

int lbm_color_step(lbm_color* c, int n) {
    int rc = center(c);
    if (rc) return rc;
    if (n < 0) return cfail(c, LBM_EINVAL, "n must be >= 0");
    for (int k = 0; k < n; ++k)
        if ((rc = cstep_once(c))) return rc;
    c->steps += n;
    return LBM_OK;
}

int lbm_color_get_fields(lbm_color* c, double* rho, double* ux, double* uy, double* uz, double* phi) {
    int rc = center(c);
    if (rc) return rc;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    const unsigned nb = (unsigned)((c->L.n + lbm::kCB - 1) / lbm::kCB);
    double* d = nullptr;
    COLOR_CUDA(c, cudaMalloc(&d, 5 * ncell * sizeof(double)));
    cudaError_t e = cudaMemsetAsync(d, 0, 5 * ncell * sizeof(double), c->stream);
    // refresh phi from the current A, B (phi of the last pre-pass lags by one step)
    if (e == cudaSuccess)
        e = cdispatch(c->prec, [&](auto zero) {
            using T = decltype(zero);
            lbm::ColorParams* none = c->d_prm;
            lbm::DevLattice L0 = c->L;
            L0.a_in = 0;  // no inlet reduction in this refresh
            lbm::k_color_pre<T><<<nb, lbm::kCB, 0, c->stream>>>((const T*)c->f[c->cur], (T*)c->A[c->cur],
                                                               (T*)c->B[c->cur], (T*)c->phi, L0, none,
                                                               c->d_partials, c->d_counter);
            lbm::k_color_export<T><<<nb, lbm::kCB, 0, c->stream>>>((const T*)c->f[c->cur], (const T*)c->phi, c->L,
                                                                  c->d_voxel, d, d + ncell, d + 2 * ncell,
                                                                  d + 3 * ncell, d + 4 * ncell);
            return cudaGetLastError();
        });
    double* outs[5] = {rho, ux, uy, uz, phi};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (outs[k]) e = cudaMemcpyAsync(outs[k], d + k * ncell, ncell * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cfail(c, LBM_ECUDA, "lbm_color_get_fields: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_color_get_flux(lbm_color* c, int face, double* Q, double* rho_bc) {
    int rc = center(c);
    if (rc) return rc;
    if (face != LBM_FACE_ZMIN && face != LBM_FACE_ZMAX) return cfail(c, LBM_EINVAL, "unknown face");
    const unsigned nb = (unsigned)((c->L.n + lbm::kCB - 1) / lbm::kCB);
    cudaError_t e = cdispatch(c->prec, [&](auto zero) {
        using T = decltype(zero);
        lbm::k_color_face_flux<T><<<nb, lbm::kCB, 0, c->stream>>>((const T*)c->f[c->cur], c->L,
                                                                 face == LBM_FACE_ZMIN ? 0 : 1, c->d_partials,
                                                                 c->d_counter2, c->d_out);
        return cudaGetLastError();
    });
    COLOR_CUDA(c, e);
    double q = 0;
    lbm::ColorParams prm{};
    COLOR_CUDA(c, cudaMemcpyAsync(&q, c->d_out, sizeof q, cudaMemcpyDeviceToHost, c->stream));
    COLOR_CUDA(c, cudaMemcpyAsync(&prm, c->d_prm, sizeof prm, cudaMemcpyDeviceToHost, c->stream));
    COLOR_CUDA(c, cudaStreamSynchronize(c->stream));
    if (Q) *Q = q;
    if (rho_bc) *rho_bc = 1.0 + (face == LBM_FACE_ZMIN ? prm.drho_in : prm.drho_out);
    return LBM_OK;
}

int lbm_color_destroy(lbm_color* c) {
    if (!c) return LBM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    crelease(c);
    delete c;
    return LBM_OK;
}

const char* lbm_color_last_error(const lbm_color* c) { return c ? c->err.c_str() : lbm::g_color_err.c_str(); }

}  // extern "C"
