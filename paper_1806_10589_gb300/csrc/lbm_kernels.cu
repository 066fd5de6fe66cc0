// CUDA kernels of the D3Q19 flux-boundary step (sm_103a).
//
//   k_step          one full time step for every pore node: pull streaming with
//                   halfway bounce-back (Eq. LBE), the Appendix B closures at the
//                   inlet/outlet planes with the inlet density of Eq. (potential),
//                   collision (Appendix A) and the store.  The same launch also
//                   forms the NEXT step's inlet density: every stored value that
//                   the next step pulls into an inlet node's known sum (Eq.
//                   inlet) is added, in FP64, by the node that produces it, then
//                   a deterministic last-block finish writes drho_in[slot ^ 1].
//   k_inlet_reduce  the same density by a pull over the inlet plane, for states
//                   set from outside a step (creation, set_*, a new Q).
//   k_step_aa       the same step on ONE buffer (AA pattern, FP64/FP32), with
//                   the layout swaps k_aa_swap / k_aa_unstream around a call.
//   k_monitors      FP64 mass / flux / max|u| / NaN reductions of a state.
//   k_export, k_init_eq, k_encode, k_decode   field and state conversions.
#include <algorithm>
#include <cstdlib>
#include <utility>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kBlock = 256;
constexpr int kReduceBlock = 256;
// Resident 256-thread blocks per SM the step kernel is compiled for (caps its
// registers at 65536 / (256 * n)); FP64 arithmetic is left unconstrained.
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 4
#endif
template <class S>
constexpr int step_min_blocks() {
    return sizeof(typename S::M) == 8 ? 1 : LBM_STEP_MIN_BLOCKS;
}

template <int... Qs, class F>
__device__ __forceinline__ void for_q(std::integer_sequence<int, Qs...>, F&& f) {
    (f(std::integral_constant<int, Qs>{}), ...);
}
using AllQ = std::make_integer_sequence<int, 19>;
template <int Q>
using qc_t = std::integral_constant<int, Q>;

// Reference profile of the 16-bit formats at the plane of padded voxel p, and
// its slope (both 0 for the formats that store d directly).
template <class S>
__device__ __forceinline__ typename S::M own_ref(const BcState* bc, const DevLattice& L, int64_t p) {
    using M = typename S::M;
    if constexpr (S::kRef) return ref_at<M>(bc, plane_of((uint64_t)p, L.sz_magic));
    else return M(0);
}
template <class S>
__device__ __forceinline__ typename S::M own_slope(const BcState* bc) {
    using M = typename S::M;
    if constexpr (S::kRef) return ref_slope<M>(bc);
    else return M(0);
}

// ---------------------------------------------------- step-kernel access ---
// Per-direction row pointers of the two distribution buffers, passed as kernel
// parameters: every gather address is one multiply-add with a constant-bank
// operand, and no register is spent on 19 hoisted row bases.
template <class T>
struct StepPtrs {
    const T* in[19];
    T* out[19];
};

// The per-node kernel forms the next step's inlet contribution from the
// registers (FP32/FP64: measured faster) or by reloading the values it has just
// stored (16-bit formats: frees the decode state, measured faster).
// LBM_CONTRIB_RELOAD = 0 / 1 forces one way for every format.
template <class S>
__host__ __device__ constexpr bool contrib_reload() {
#ifdef LBM_CONTRIB_RELOAD
    return LBM_CONTRIB_RELOAD != 0;
#else
    return S::kRef;
#endif
}

// LBM_L2_HINTS: 0 = no hints; 1 = index structures evict-last; 2 = also the
// distribution streams evict-first.
#ifndef LBM_L2_HINTS
#define LBM_L2_HINTS 1
#endif

template <class T>
__device__ __forceinline__ T ld_index(const T* a, uint64_t pol) {
#if LBM_L2_HINTS >= 1
    return ld_hint(a, pol);
#else
    (void)pol;
    return __ldg(a);
#endif
}
template <class T>
__device__ __forceinline__ T ld_stream(const T* a, uint64_t pol) {
#if LBM_L2_HINTS >= 2
    return ld_hint(a, pol);
#else
    (void)pol;
    return __ldg(a);
#endif
}
template <class T>
__device__ __forceinline__ void st_stream(T* a, T v, uint64_t pol) {
#if LBM_L2_HINTS >= 2
    st_hint(a, v, pol);
#else
    (void)pol;
    *a = v;
#endif
}

// Pull all 19 values of node i (padded voxel p): a pore source gives its own
// value, a solid or outside source the node's opposite value (halfway
// bounce-back; the z-outside ones are replaced by the closure).
template <class S, bool OFF32 = false>
__device__ __forceinline__ void pull_step(typename S::M* d, const StepPtrs<typename S::T>& P,
                                          const DevLattice& L, uint32_t p, int i, uint64_t pol_f,
                                          uint64_t pol_idx, typename S::M r_own, typename S::M g) {
    using M = typename S::M;
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        if constexpr (Q == 0) {
            d[0] = S::template dec<0>(ld_stream(P.in[0] + i, pol_f), r_own);
        } else {
            // padded voxel indices fit in 32 bits (checked at creation)
            const int id = ld_index(L.grid + (uint32_t)(p + (uint32_t)L.goff[Q]), pol_idx);
            const typename S::T* a;
            if constexpr (OFF32)  // row 0 plus one 32-bit element offset (rows are ns apart)
                a = P.in[0] + (id >= 0 ? (uint32_t)Q * (uint32_t)L.ns + (uint32_t)id
                                       : (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)i);
            else
                a = id >= 0 ? P.in[Q] + id : P.in[opp(Q)] + i;
            // a pulled value was written on plane z - xi_z (reference r_own - g xi_z)
            const M r = (cz(Q) != 0 && id >= 0) ? r_own - M(cz(Q)) * g : r_own;
            d[Q] = S::template dec<Q>(ld_stream(a, pol_f), r);
        }
    });
}

template <class S>
__device__ __forceinline__ void store_step(const typename S::M* d, const StepPtrs<typename S::T>& P,
                                           int i, uint64_t pol_f, typename S::M r_own, uint32_t seed) {
    encode_node<S>(d, seed, i, [&](auto) { return r_own; }, [&](auto qc, typename S::T v) {
        constexpr int Q = decltype(qc)::value;
        st_stream(P.out[Q] + i, v, pol_f);
    });
}

// Stochastic-rounding seed of this step (16-bit formats), and the next one.
template <class S>
__device__ __forceinline__ uint32_t step_seed(const BcState* bc, int slot) {
    if constexpr (S::kRef) return bc->sr_seed[slot];
    else return 0u;
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
// Warp sums in the storage's arithmetic type (FP32 for the FP32/16-bit
// formats): FP64 arithmetic is scarce on GB300, so per-node values and the
// first 32-way level stay in M and only the block level runs in FP64.
template <class M>
__device__ __forceinline__ M warp_sum_m(M v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
template <class M>
__device__ __forceinline__ M warp_max_m(M v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const M w = __shfl_down_sync(0xffffffffu, v, o);  // every lane shuffles, then compares
        v = v > w ? v : w;
    }
    return v;
}
template <int NT, class M>
__device__ __forceinline__ double block_sum_m(M v, double* sh) {
    v = warp_sum_m(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;  // valid in thread 0
}
template <int NT, class M>
__device__ __forceinline__ double block_max_m(M v, double* sh) {
    v = warp_max_m(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
        r = warp_max(r);
    }
    __syncthreads();
    return r;
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
k_inlet_reduce(const typename S::T* __restrict__ fin, int slot, DevLattice L, BcState* bc,
               double* __restrict__ partials, unsigned* __restrict__ counter) {
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i64 = (int64_t)blockIdx.x * kReduceBlock + threadIdx.x;
    double k = 0.0;
    if (i64 < L.a_in) {
        const int i = (int)i64;
        const int64_t p = L.vox[i];
        using M = typename S::M;
        const M r_own = own_ref<S>(bc, L, p), g = own_slope<S>(bc);
        M d[19];
        for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 6, 7, 8, 9, 10, 12, 13, 16, 17>{},
              [&](auto qc) {
                  constexpr int Q = decltype(qc)::value;
                  d[Q] = pull<S, Q>(fin, L.ns, L.grid, p, i, L.sy, L.sz, r_own, g);
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
        bc->drho_in[slot] = (bc->Q + s) / (double)L.a_in;
        *counter = 0u;
    }
}

// ---------------------------------------------------------- the step ---
// Contribution of pore node i (on plane z = 0 or z = 1) to the next step's
// inlet known sum S' = sum over inlet nodes of K'.  A value stored in direction
// p lands, at the next pull, on node i + xi_p (if that is a pore) or bounces
// back to i as direction opp(p).  It enters S' when it lands on the plane z = 0
// in a direction with xi_z = 0 (weight 1) or xi_z = -1 (weight 2):
//   z = 0:  all xi_z = 0 values (they stay on the plane either way), plus twice
//           each xi_z = +1 value whose destination on z = 1 is solid;
//   z = 1:  twice each xi_z = -1 value whose destination on z = 0 is a pore.
// `val(Q)` returns the stored value of direction Q exactly as the next step
// will decode it.
template <class S, class V>
__device__ __forceinline__ double inlet_contribution(const DevLattice& L, uint32_t p, int i, V&& val) {
    double s = 0.0;
    auto dest_is_pore = [&](auto qc) -> bool {
        constexpr int Q = decltype(qc)::value;  // destination i + xi_Q = pull source of opp(Q)
        return __ldg(L.grid + (uint32_t)(p + (uint32_t)L.goff[opp(Q)])) >= 0;
    };
    if (i < L.a_in) {
        for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 7, 8, 9, 10>{},
              [&](auto qc) { s += val(qc); });
        for_q(std::integer_sequence<int, 5, 11, 14, 15, 18>{},
              [&](auto qc) { if (!dest_is_pore(qc)) s += 2.0 * val(qc); });
    } else {
        for_q(std::integer_sequence<int, 6, 12, 13, 16, 17>{},
              [&](auto qc) { if (dest_is_pore(qc)) s += 2.0 * val(qc); });
    }
    return s;
}

// From values still in registers (the pipelined kernel).
template <class S>
__device__ __forceinline__ double next_inlet_part(const typename S::M* d, const DevLattice& L,
                                                  int64_t p, int i, typename S::M r_own, uint32_t seed) {
    return inlet_contribution<S>(L, (uint32_t)p, i, [&](auto qc) -> double {
        constexpr int Q = decltype(qc)::value;
        return (double)S::template dec<Q>(S::template enc_sr<Q>(d[Q], r_own, sr_key<S>(seed, i, Q)), r_own);
    });
}

// From the values this thread has just stored (the per-node kernel): the
// registers of the collision are free again, and only the ~2 % of nodes on the
// planes next to the inlet pay the reload.
template <class S>
__device__ __forceinline__ double next_inlet_part_stored(const StepPtrs<typename S::T>& P, const DevLattice& L,
                                                         uint32_t p, int i, typename S::M r_own) {
    return inlet_contribution<S>(L, p, i, [&](auto qc) -> double {
        constexpr int Q = decltype(qc)::value;
        const typename S::T v = *(volatile const typename S::T*)(P.out[Q] + i);
        return (double)S::template dec<Q>(v, r_own);
    });
}

// LBM_STEP_PREFETCH: each block asks L2 (a bulk prefetch, nothing waited for)
// for the 19 input rows and the voxel list of the block that many blocks ahead,
// as the gather-scatter AA step does; 0 = off.  Measured on the 256^3 pack
// (same-call A/B, bitwise equal states): FP32 step 0.1953 ms without, 0.1764,
// 0.1745 and 0.1773 ms at 128, 224 and 320 blocks ahead; FP16-dev 0.1730,
// 0.1640, 0.1620 and 0.1614 ms.
#ifndef LBM_STEP_PREFETCH
#define LBM_STEP_PREFETCH 224
#endif

// OFF32: pulls addressed as row 0 plus a 32-bit element offset (buffers of
// 19 ns < 2^32 elements), as in the gather-scatter AA step.
template <class S, bool OFF32 = false>
__global__ void __launch_bounds__(kBlock, step_min_blocks<S>())
k_step(const StepPtrs<typename S::T> P, int slot, DevLattice L, typename S::M sp, typename S::M sm,
       BcState* bc, double* __restrict__ partials, unsigned* __restrict__ counter) {
    using M = typename S::M;
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i64 = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int i = (int)i64;
    double part = 0.0;
    if constexpr (LBM_STEP_PREFETCH > 0) {
        // threads 0..18: input row q (rows are P.in[0] + q ns; the 128-element
        // padding keeps every range 16-byte aligned); thread 19: the voxel list,
        // cut to a multiple of 4 entries
        const int64_t s = ((int64_t)blockIdx.x + LBM_STEP_PREFETCH) * kBlock;
        const int t = (int)threadIdx.x;
        if (t < 19) l2_prefetch_range(P.in[0] + (int64_t)t * L.ns, s, kBlock, L.ns);
        else if (t == 19) l2_prefetch_range(L.vox, s, kBlock, L.n & ~(int64_t)3);
    }
    if (i64 < L.n) {
#if LBM_L2_HINTS >= 2
        const uint64_t pol_f = l2_policy_evict_first();
#else
        const uint64_t pol_f = 0;
#endif
#if LBM_L2_HINTS >= 1
        const uint64_t pol_idx = l2_policy_evict_last();
#else
        const uint64_t pol_idx = 0;
#endif
        const uint32_t p = ld_index(L.vox + i, pol_idx);
        const M r_own = own_ref<S>(bc, L, p), g = own_slope<S>(bc);
        const uint32_t seed = step_seed<S>(bc, slot);
        M d[19];
        pull_step<S, OFF32>(d, P, L, p, i, pol_f, pol_idx, r_own, g);
        if (i < L.a_in) {
            // Section 2: after streaming, before collision.  u_z from Eq. (inlet)
            // with the density of Eq. (potential); then the Appendix B closure.
            const M drin = bc->inlet_mode ? M(bc->drho_in_fixed) : M(bc->drho_in[slot]);
            close_inlet(d, drin - inlet_known(d));
        } else if (i64 >= L.n - L.a_out) {
            const M uz = outlet_known(d) - M(bc->drho_out);
            close_outlet(d, uz);
        }
        collide(d, sp, sm);
        store_step<S>(d, P, i, pol_f, r_own, seed);
        if (i64 < L.a_01) {
            if constexpr (contrib_reload<S>()) part = next_inlet_part_stored<S>(P, L, p, i, r_own);
            else part = next_inlet_part<S>(d, L, p, i, r_own, seed);
        }
    }
    // blocks that hold plane z = 0 or z = 1 nodes (block-uniform branch)
    if ((int64_t)blockIdx.x * kBlock < L.a_01) {
        const unsigned nb = (unsigned)((L.a_01 + kBlock - 1) / kBlock);
        const double b = block_sum<kBlock>(part, sh);
        if (threadIdx.x == 0) {
            partials[blockIdx.x] = b;
            __threadfence();
            last = atomicAdd(counter, 1u) == nb - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            double s = 0.0;
            for (unsigned j = threadIdx.x; j < nb; j += kBlock) s += __ldcg(partials + j);
            s = block_sum<kBlock>(s, sh);
            if (threadIdx.x == 0) {
                bc->drho_in[slot ^ 1] = (bc->Q + s) / (double)L.a_in;
                if constexpr (S::kRef) bc->sr_seed[slot ^ 1] = sr_next(bc->sr_seed[slot]);
                *counter = 0u;
            }
        }
    }
}

// ------------------------------------------------------ AA-pattern step ---
// Single-buffer variant (every storage format).  At rest the state has the pull
// layout of k_step, F[q][x] = f*_q(x) (post-collision values at their own node).
// The library first swaps every node's opposite pairs (layout S:
// F[opp q][x] = f*_q(x)), then alternates
//   odd step:  in_q(x) = F[opp q][x - xi_q] for a pore source, else F[q][x]
//              (halfway bounce-back); closures, collision; f*_q(x) goes to
//              F[q][x + xi_q] for a pore destination, else to F[opp q][x]
//              (layout S -> I, I[q][x] = the value arriving at x in direction q);
//   even step: in_q(x) = F[q][x]; closures, collision; f*_q(x) -> F[opp q][x]
//              (layout I -> S);
// and swaps the pairs back before anything else reads the state (after an odd
// count, k_aa_unstream first turns layout I into S); consecutive step calls stay
// in the in-place layouts.  Within a step every slot is read and then written by
// one node only, so the update runs in place.  Values leaving through the z
// faces are kept like bounced ones; the closures overwrite them.  The next
// step's inlet density is formed exactly as in k_step: the landing rule of a
// post-collision value does not depend on where it is stored.
// Where the gather-scatter step keeps its 18 neighbour ids across the
// collision (LBM_AA_IDS): 0 = registers (spills at the 64-register cap),
// 1 = loads them again from the id grid, 2 = shared memory (18 KB per block;
// with LBM_AA_SMEM_OFF the gather offsets instead of the ids).  Measured best:
// 2 for every format (LBM_AA16_IDS for the 16-bit ones); with ids instead of
// offsets staged, 1 and 2 were equal in FP32.
#ifndef LBM_AA_IDS
#define LBM_AA_IDS 2
#endif
#ifndef LBM_AA16_IDS
#define LBM_AA16_IDS 2
#endif


// Row pointers of the single buffer as kernel parameters (constant bank), as
// for k_step: no registers spent on 19 row addresses.
template <class T>
struct AAPtrs {
    T* row[19];
};

// Resident blocks per SM the two AA kernels are compiled for (register caps).
// The FP32 gather-scatter step measured best at 5 (48 registers): with the
// gather offsets staged in shared memory it compiles there without spills, and
// its launch took 0.1897 ms against 0.1970 ms at 4 (64 registers).  (With the
// ids reloaded for the scatter, 4 was best with the L2 prefetch, 5 with spills
// without it.)
#ifndef LBM_AA_MIN_BLOCKS
#define LBM_AA_MIN_BLOCKS 5
#endif
#ifndef LBM_AA_EVEN_MIN_BLOCKS
#define LBM_AA_EVEN_MIN_BLOCKS 6
#endif
// LBM_AA_ID_HINT: 1 = the id grid is read with the L2 evict-last policy, 0 = plain.
#ifndef LBM_AA_ID_HINT
#define LBM_AA_ID_HINT 1
#endif
// The 16-bit formats carry the reference profile and the rounding seed too.
#ifndef LBM_AA16_MIN_BLOCKS
#define LBM_AA16_MIN_BLOCKS 5
#endif
#ifndef LBM_AA16_EVEN_MIN_BLOCKS
#define LBM_AA16_EVEN_MIN_BLOCKS 5
#endif
// LBM_AA_PREFETCH: the FP32/FP64 gather-scatter step asks L2 for the rows of the
// block that many blocks ahead (a bulk prefetch, nothing waited for), so that
// the DRAM requests in flight no longer depend on how many warps are waiting on
// their own gathers; 0 = off.  Measured on the 256^3 pack: the gain is flat from
// about 160 to 288 blocks ahead and falls off outside; at 224 the AA step pair is
// 4.7 % shorter than without (with the cap of 4 blocks).
#ifndef LBM_AA_PREFETCH
#define LBM_AA_PREFETCH 224
#endif
// LBM_AA16_PREFETCH: the same bulk L2 prefetch for the 16-bit gather-scatter
// step, that many blocks ahead; 0 = off.  Measured on the 256^3 pack: FP16-dev
// step 0.1735 against 0.1763 ms without, BF16-dev 0.1742 against 0.1826 ms (a
// 4-block register cap or reloaded ids with it were 10-14 % slower).
#ifndef LBM_AA16_PREFETCH
#define LBM_AA16_PREFETCH 224
#endif
// LBM_AA16_PAIR_SCATTER: 1 = the 16-bit gather-scatter step rounds each
// opposite pair with one conversion before its two stores, 0 = one conversion
// per value next to its store.  Measured on the 256^3 pack: 0 is 2.9 % (FP16)
// and 2.8 % (BF16) faster in that launch (the node-local launch rounds pairs).
#ifndef LBM_AA16_PAIR_SCATTER
#define LBM_AA16_PAIR_SCATTER 0
#endif
template <class S, bool ODD>
constexpr int aa_min_blocks() {
    if constexpr (sizeof(typename S::M) == 8) return 1;
    else if constexpr (S::kRef) return ODD ? LBM_AA16_MIN_BLOCKS : LBM_AA16_EVEN_MIN_BLOCKS;
    else return ODD ? LBM_AA_MIN_BLOCKS : LBM_AA_EVEN_MIN_BLOCKS;
}
template <class T>
__device__ __forceinline__ T ld_aa_index(const T* a, uint64_t pol) {
#if LBM_AA_ID_HINT
    return ld_index(a, pol);
#else
    (void)pol;
    return __ldg(a);
#endif
}
__device__ __forceinline__ uint64_t aa_index_policy() {
#if LBM_AA_ID_HINT
    return l2_policy_evict_last();
#else
    return 0;
#endif
}

// LBM_AA_SMEM_OFF: 1 = with ids staged in shared memory (LBM_AA16_IDS /
// LBM_AA_IDS 2) and 32-bit offsets, the gather stores each direction's element
// offset instead of its id.  The scatter destination of q is the gather source
// of opp(q) -- F[q][x + xi_q] for a pore there, else the bounce-back slot
// F[opp q][x], both read by the gather of opp(q) -- so the scatter reads its
// offset as it is and needs no id test or offset arithmetic; 0 = ids staged.
// Measured on the 256^3 pack (same-call A/B, bitwise equal states): the
// gather-scatter launch 0.2006 -> 0.1825 ms (FP16-dev), 0.2024 -> 0.1840 ms
// (BF16-dev), and with the FP32 ids staged as well (LBM_AA_IDS 2; staged ids
// alone gave 0.2007 ms) 0.2013 -> 0.1972 ms.
#ifndef LBM_AA_SMEM_OFF
#define LBM_AA_SMEM_OFF 1
#endif

// OFF32 (gather-scatter launch, buffers of 19 ns < 2^32 elements): every
// neighbour address is row 0 plus one 32-bit element offset, the source or
// destination row chosen by a 32-bit select, instead of a select between two
// 64-bit row pointers.  Measured on the 256^3 pack: the launch 6.5 % (FP32) and
// 8 % (FP16-dev) shorter.
template <class S, bool ODD, bool OFF32 = false>
__global__ void __launch_bounds__(kBlock, aa_min_blocks<S, ODD>())
k_step_aa(const AAPtrs<typename S::T> F, int slot, DevLattice L, typename S::M sp, typename S::M sm,
          BcState* bc, double* __restrict__ partials, unsigned* __restrict__ counter) {
    using M = typename S::M;
    __shared__ double sh[32];
    __shared__ bool last;
    constexpr int kIds = S::kRef ? LBM_AA16_IDS : LBM_AA_IDS;
    // staged per direction: the gather's element offset (kOffs) or the pore id
    constexpr bool kOffs = OFF32 && kIds == 2 && LBM_AA_SMEM_OFF;
    __shared__ int sid[(ODD && kIds == 2) ? 18 : 1][kBlock];
    const int64_t i64 = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int i = (int)i64;
    double part = 0.0;
    constexpr int kAhead = S::kRef ? LBM_AA16_PREFETCH : LBM_AA_PREFETCH;
    if constexpr (ODD && kAhead > 0) {
        // threads 0..18: row q of the buffer (rows are F.row[0] + q ns, as
        // launched; 128-element padding keeps every range 16-byte aligned for
        // 2-byte values too); thread 19: the voxel list, cut to a multiple of 4 entries
        const int64_t s = ((int64_t)blockIdx.x + kAhead) * kBlock;
        const int t = (int)threadIdx.x;
        if (t < 19) l2_prefetch_range(F.row[0] + (int64_t)t * L.ns, s, kBlock, L.ns);
        else if (t == 19) l2_prefetch_range(L.vox, s, kBlock, L.n & ~(int64_t)3);
    }
    if (i64 < L.n) {
        M d[19];
        int nb[19];  // odd step: pore id of x - xi_q (the pull source of q), or a negative marker
        // 16-bit formats: every stored value is encoded with the reference of the
        // plane of the node that holds it (the even step writes its own slots; the
        // odd step encodes a scattered value with its destination's plane), so a
        // value read from the neighbour x - xi_q decodes with r(z - xi_z).
        M r_own = M(0), g = M(0);
        const uint32_t seed = step_seed<S>(bc, slot);
        if constexpr (ODD) {
            const uint64_t pol_idx = aa_index_policy();
            const uint32_t p = ld_aa_index(L.vox + i, pol_idx);
            r_own = own_ref<S>(bc, L, p);
            g = own_slope<S>(bc);
            d[0] = S::template dec<0>(F.row[0][i], r_own);
            for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value + 1;
                nb[Q] = ld_aa_index(L.grid + (uint32_t)(p + (uint32_t)L.goff[Q]), pol_idx);
                if constexpr (kIds == 2 && !kOffs) sid[Q - 1][threadIdx.x] = nb[Q];
                if constexpr (S::kRef) {
                    // 16-bit (instruction-bound): one load and one decode, the
                    // source slot and its plane selected
                    const bool pore = nb[Q] >= 0;
                    const typename S::T* src;
                    if constexpr (OFF32) {  // one 32-bit element offset from row 0 (the rows are ns apart)
                        const uint32_t off = pore ? (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)nb[Q]
                                                  : (uint32_t)Q * (uint32_t)L.ns + (uint32_t)i;
                        if constexpr (kOffs) sid[Q - 1][threadIdx.x] = (int)off;
                        src = F.row[0] + off;
                    } else {
                        src = pore ? F.row[opp(Q)] + nb[Q] : F.row[Q] + i;
                    }
                    d[Q] = S::template dec<Q>(*src, pore ? r_own - M(cz(Q)) * g : r_own);
                } else {
                    if constexpr (OFF32) {
                        const uint32_t off = nb[Q] >= 0 ? (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)nb[Q]
                                                        : (uint32_t)Q * (uint32_t)L.ns + (uint32_t)i;
                        if constexpr (kOffs) sid[Q - 1][threadIdx.x] = (int)off;
                        d[Q] = F.row[0][off];
                    } else {
                        d[Q] = nb[Q] >= 0 ? F.row[opp(Q)][nb[Q]] : F.row[Q][i];
                    }
                }
            });
        } else {
            if constexpr (S::kRef) r_own = own_ref<S>(bc, L, __ldg(L.vox + i));
            for_q(AllQ{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value;
                d[Q] = S::template dec<Q>(F.row[Q][i], r_own);
            });
        }
        if (i < L.a_in) {
            const M drin = bc->inlet_mode ? M(bc->drho_in_fixed) : M(bc->drho_in[slot]);
            close_inlet(d, drin - inlet_known(d));
        } else if (i64 >= L.n - L.a_out) {
            close_outlet(d, outlet_known(d) - M(bc->drho_out));
        }
        collide(d, sp, sm);
        // an opaque copy of i for the stores: sharing the load addresses would keep
        // 19 64-bit addresses live across the collision
        int j;
        asm volatile("mov.b32 %0, %1;" : "=r"(j) : "r"(i));
        if constexpr (ODD) {
            // kIds == 1: fresh policy and voxel index, nothing of the gather stays live
            const uint64_t pol_s = kIds == 1 ? aa_index_policy() : 0;
            const uint32_t ps = kIds == 1 ? ld_aa_index(L.vox + j, pol_s) : 0u;
            F.row[0][j] = S::template enc_sr<0>(d[0], r_own, sr_key<S>(seed, i, 0));
            // x + xi_Q is the pull source of opp(Q)
            auto dest = [&](auto qc) -> int {
                constexpr int Q = decltype(qc)::value;
                if constexpr (kIds == 1) return ld_aa_index(L.grid + (uint32_t)(ps + (uint32_t)L.goff[opp(Q)]), pol_s);
                else if constexpr (kIds == 2) return sid[opp(Q) - 1][threadIdx.x];
                else return nb[opp(Q)];
            };
            if constexpr (kOffs) {
                // the destination of Q is the gather source of opp(Q), its offset
                // staged by this thread; a pore destination lies in row Q, a
                // bounce-back one in row opp(Q)
                for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                    constexpr int Q = decltype(qc)::value + 1;
                    const uint32_t off = (uint32_t)sid[opp(Q) - 1][threadIdx.x];
                    if constexpr (S::kRef) {
                        M r = r_own;
                        if constexpr (cz(Q) != 0) {
                            const bool pore = (Q & 1) ? off < (uint32_t)(Q + 1) * (uint32_t)L.ns
                                                      : off >= (uint32_t)Q * (uint32_t)L.ns;
                            r = pore ? r_own + M(cz(Q)) * g : r_own;
                        }
                        F.row[0][off] = S::template enc_sr<Q>(d[Q], r, sr_key<S>(seed, i, Q));
                    } else {
                        F.row[0][off] = d[Q];
                    }
                });
            } else if constexpr (S::kRef && !LBM_AA16_PAIR_SCATTER) {
                for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                    constexpr int Q = decltype(qc)::value + 1;
                    const int dst = dest(qc_t<Q>{});
                    const bool pore = dst >= 0;
                    typename S::T* out;
                    if constexpr (OFF32)
                        out = F.row[0] + (pore ? (uint32_t)Q * (uint32_t)L.ns + (uint32_t)dst
                                               : (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)j);
                    else
                        out = pore ? F.row[Q] + dst : F.row[opp(Q)] + j;
                    *out = S::template enc_sr<Q>(d[Q], pore ? r_own + M(cz(Q)) * g : r_own, sr_key<S>(seed, i, Q));
                });
            } else if constexpr (S::kRef) {
                // 16-bit: per opposite pair one stochastic conversion; per value one
                // store, destination slot and plane selected
                for_q(std::make_integer_sequence<int, 9>{}, [&](auto pc) {
                    constexpr int Q = 2 * decltype(pc)::value + 1;
                    const int dq = dest(qc_t<Q>{});
                    const int dq1 = dest(qc_t<Q + 1>{});
                    const uint32_t h = S::template enc_sr2<Q>(d[Q], dq >= 0 ? r_own + M(cz(Q)) * g : r_own, d[Q + 1],
                                                              dq1 >= 0 ? r_own - M(cz(Q)) * g : r_own,
                                                              sr_key<S>(seed, i, Q), sr_key<S>(seed, i, Q + 1));
                    *(dq >= 0 ? F.row[Q] + dq : F.row[Q + 1] + j) = S::half_of(h, true);
                    *(dq1 >= 0 ? F.row[Q + 1] + dq1 : F.row[Q] + j) = S::half_of(h, false);
                });
            } else {  // FP32/FP64 store d directly; the branch form measured faster there
                for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                    constexpr int Q = decltype(qc)::value + 1;
                    const int dst = dest(qc_t<Q>{});
                    if constexpr (OFF32) {
                        F.row[0][dst >= 0 ? (uint32_t)Q * (uint32_t)L.ns + (uint32_t)dst
                                          : (uint32_t)opp(Q) * (uint32_t)L.ns + (uint32_t)j] = d[Q];
                    } else {
                        if (dst >= 0) F.row[Q][dst] = d[Q];
                        else F.row[opp(Q)][j] = d[Q];
                    }
                });
            }
        } else {
            encode_node<S>(d, seed, i, [&](auto) { return r_own; }, [&](auto qc, typename S::T v) {
                constexpr int Q = decltype(qc)::value;
                F.row[opp(Q)][j] = v;
            });
        }
        if (i64 < L.a_01) {
            // the counted values land on plane 0: from plane 1 (xi_z = -1, stored
            // with plane 0's reference in the odd step) or staying on plane 0
            part = inlet_contribution<S>(L, L.vox[i], i, [&](auto qc) -> double {
                constexpr int Q = decltype(qc)::value;
                const M rq = (ODD && cz(Q) < 0) ? r_own - g : r_own;
                return (double)S::template dec<Q>(S::template enc_sr<Q>(d[Q], rq, sr_key<S>(seed, i, Q)), rq);
            });
        }
    }
    if ((int64_t)blockIdx.x * kBlock < L.a_01) {
        const unsigned nbk = (unsigned)((L.a_01 + kBlock - 1) / kBlock);
        const double b = block_sum<kBlock>(part, sh);
        if (threadIdx.x == 0) {
            partials[blockIdx.x] = b;
            __threadfence();
            last = atomicAdd(counter, 1u) == nbk - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            double s = 0.0;
            for (unsigned j = threadIdx.x; j < nbk; j += kBlock) s += __ldcg(partials + j);
            s = block_sum<kBlock>(s, sh);
            if (threadIdx.x == 0) {
                bc->drho_in[slot ^ 1] = (bc->Q + s) / (double)L.a_in;
                if constexpr (S::kRef) bc->sr_seed[slot ^ 1] = sr_next(bc->sr_seed[slot]);
                *counter = 0u;
            }
        }
    }
}

// Pull layout <-> layout S: swap F[q][x] and F[opp q][x] at every node.
// All 18 loads are issued before any store (the rows of one buffer could alias
// as far as the compiler knows, which would serialise load-store pairs).
template <class T>
__global__ void k_aa_swap(T* __restrict__ f, int64_t n, int64_t ns) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T v[19];
#pragma unroll
    for (int q = 1; q < 19; ++q) v[q] = f[(int64_t)q * ns + i];
#pragma unroll
    for (int q = 1; q < 19; q += 2) {  // opposite pairs are (q, q + 1), q odd
        f[(int64_t)q * ns + i] = v[q + 1];
        f[(int64_t)(q + 1) * ns + i] = v[q];
    }
}

// Layout I -> layout S after an odd step: the value that arrived at x in
// direction q from the pore x - xi_q belongs in F[opp q][x - xi_q], and that
// slot holds the value that arrived at x - xi_q in direction opp q from x,
// which belongs in F[q][x]: one swap per pair, done by the node with odd q.
// A value that arrived by bounce-back is already in place.
// 16-bit formats: a moved value is re-encoded from its old holder's plane to
// the new one's (opposite directions share the weight).
template <class S>
__global__ void k_aa_unstream(typename S::T* __restrict__ f, DevLattice L, const BcState* bc) {
    using T = typename S::T;
    using M = typename S::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const uint32_t p = L.vox[i];
    const M r_own = own_ref<S>(bc, L, p), g = own_slope<S>(bc);
    // ids and values first, stores after (see k_aa_swap)
    int id[19];
    T ta[19], tb[19];
    for_q(std::integer_sequence<int, 1, 3, 5, 7, 9, 11, 13, 15, 17>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        id[Q] = __ldg(L.grid + (uint32_t)(p + (uint32_t)L.goff[Q]));
    });
    for_q(std::integer_sequence<int, 1, 3, 5, 7, 9, 11, 13, 15, 17>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        if (id[Q] >= 0) {
            ta[Q] = f[(int64_t)Q * L.ns + i];
            tb[Q] = f[(int64_t)(Q + 1) * L.ns + id[Q]];
        }
    });
    for_q(std::integer_sequence<int, 1, 3, 5, 7, 9, 11, 13, 15, 17>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        if (id[Q] >= 0) {
            T* a = f + (int64_t)Q * L.ns + i;
            T* b = f + (int64_t)(Q + 1) * L.ns + id[Q];
            if constexpr (S::kRef) {
                const M r_src = r_own - M(cz(Q)) * g;  // plane of x - xi_Q
                *a = S::template enc<Q>(S::template dec<Q>(tb[Q], r_src), r_own);
                *b = S::template enc<Q>(S::template dec<Q>(ta[Q], r_own), r_src);
            } else {
                *a = tb[Q];
                *b = ta[Q];
            }
        }
    });
}

// ------------------------------------------------ pipelined step kernel ---
// The same step as k_step, restructured for memory-level parallelism: a
// persistent grid walks 256-node tiles (tile t, t + G, t + 2G, ...), and every
// gather goes through cp.async into shared memory one tile ahead of its use:
//   A(t): the 18 neighbour ids of tile t        (id grid -> smem, L2 evict-last)
//   B(t): the 19 pulled values of tile t         (distributions -> smem)
// While tile t is collided, B(t + G) and A(t + 2G) are in flight, so the loads
// outstanding per SM no longer cost registers.  Each thread only reads back the
// shared-memory slots its own copies filled, so the pipeline needs no barrier.
// 16-bit values are fetched as the aligned 4-byte pair that contains them.

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(unsigned dst, const void* src) {
    if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_hint4(unsigned dst, const void* src, uint64_t pol) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, 4, %2;" ::"r"(dst), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <class S>
struct AsyncSlot {
    using T = typename S::T;
    static constexpr int kBytes = sizeof(T) >= 4 ? (int)sizeof(T) : 4;  // bytes fetched per value
};

template <int NT>
constexpr size_t async_smem_bytes(int slot_bytes) {
    return (size_t)18 * NT * 4 + (size_t)2 * 19 * NT * slot_bytes;
}

// A(t): neighbour ids of this thread's node of tile t into ids[q-1][tid].
template <int NT>
__device__ __forceinline__ void issue_ids(int* ids, const DevLattice& L, uint32_t p, uint64_t pol) {
    for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value + 1;
        cp_async_hint4(smem_u32(ids + (Q - 1) * NT + threadIdx.x), L.grid + (int64_t)p + L.goff[Q], pol);
    });
}

// B(t): the 19 pulled values of node i into vals[q][tid]; returns the bit mask
// of 16-bit values that sit in the upper half of their fetched 4-byte pair.
template <class S, int NT>
__device__ __forceinline__ unsigned issue_vals(unsigned char* vals, const int* ids,
                                               const StepPtrs<typename S::T>& P, int i, unsigned& nbr) {
    using T = typename S::T;
    constexpr int SB = AsyncSlot<S>::kBytes;
    unsigned hi = 0;
    nbr = 0;
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        const T* a;
        if constexpr (Q == 0) {
            a = P.in[0] + i;
        } else {
            const int id = ids[(Q - 1) * NT + threadIdx.x];
            a = id >= 0 ? P.in[Q] + id : P.in[opp(Q)] + i;
            if constexpr (S::kRef && cz(Q) != 0) nbr |= (unsigned)(id >= 0) << Q;
        }
        const unsigned dst = smem_u32(vals + ((size_t)Q * NT + threadIdx.x) * SB);
        if constexpr (sizeof(T) == 2) {
            const uintptr_t u = reinterpret_cast<uintptr_t>(a);
            hi |= (unsigned)((u >> 1) & 1u) << Q;
            cp_async<4>(dst, reinterpret_cast<const void*>(u & ~(uintptr_t)3));
        } else {
            cp_async<SB>(dst, a);
        }
    });
    return hi;
}

template <class S, int NT>
__device__ __forceinline__ void read_vals(typename S::M* d, const unsigned char* vals, unsigned hi,
                                          unsigned nbr, typename S::M r_own, typename S::M g) {
    using T = typename S::T;
    using M = typename S::M;
    constexpr int SB = AsyncSlot<S>::kBytes;
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        const unsigned char* slot = vals + ((size_t)Q * NT + threadIdx.x) * SB;
        const M r = (cz(Q) != 0 && ((nbr >> Q) & 1u)) ? r_own - M(cz(Q)) * g : r_own;
        if constexpr (sizeof(T) == 2) {
            const T* pair = reinterpret_cast<const T*>(slot);
            d[Q] = S::template dec<Q>(pair[(hi >> Q) & 1u], r);
        } else {
            d[Q] = S::template dec<Q>(*reinterpret_cast<const T*>(slot), r);
        }
    });
}

template <class S, int NT>
__global__ void __launch_bounds__(NT)
k_step_async(const StepPtrs<typename S::T> P, int slot, DevLattice L, typename S::M sp,
             typename S::M sm, BcState* bc, double* __restrict__ partials,
             unsigned* __restrict__ counter) {
    using M = typename S::M;
    constexpr int SB = AsyncSlot<S>::kBytes;
    extern __shared__ __align__(16) unsigned char smem[];
    int* ids = reinterpret_cast<int*>(smem);
    unsigned char* vals0 = smem + (size_t)18 * NT * 4;
    unsigned char* vals1 = vals0 + (size_t)19 * NT * SB;
    __shared__ double sh[32];
    __shared__ bool last;

    const int64_t ntiles = (L.n + NT - 1) / NT;
    const int64_t nt01 = (L.a_01 + NT - 1) / NT;
    const int64_t G = gridDim.x;
    const uint64_t pol_idx = l2_policy_evict_last();
    auto node = [&](int64_t t) -> int64_t { return t * NT + threadIdx.x; };

    int64_t t = blockIdx.x;
    if (t >= ntiles) return;
    // prologue: A(t); wait; B(t); A(t + G)
    uint32_t p_cur = 0, p_next = 0, p_next2 = 0;
    if (node(t) < L.n) p_cur = __ldg(L.vox + node(t));
    if (t + G < ntiles && node(t + G) < L.n) p_next = __ldg(L.vox + node(t + G));
    if (t + 2 * G < ntiles && node(t + 2 * G) < L.n) p_next2 = __ldg(L.vox + node(t + 2 * G));
    if (node(t) < L.n) issue_ids<NT>(ids, L, p_cur, pol_idx);
    cp_async_commit();
    cp_async_wait_all();
    unsigned hi_cur = 0, hi_next = 0, nb_cur = 0, nb_next = 0;
    if (node(t) < L.n) hi_cur = issue_vals<S, NT>(vals0, ids, P, (int)node(t), nb_cur);
    cp_async_commit();
    if (t + G < ntiles && node(t + G) < L.n) issue_ids<NT>(ids, L, p_next, pol_idx);
    cp_async_commit();

    for (int k = 0; t < ntiles; ++k, t += G) {
        unsigned char* vcur = (k & 1) ? vals1 : vals0;
        unsigned char* vnext = (k & 1) ? vals0 : vals1;
        cp_async_wait_all();  // B(t) and A(t + G) have landed
        const int64_t tn = t + G, tn2 = t + 2 * G;
        if (tn < ntiles && node(tn) < L.n) hi_next = issue_vals<S, NT>(vnext, ids, P, (int)node(tn), nb_next);
        cp_async_commit();
        if (tn2 < ntiles && node(tn2) < L.n) issue_ids<NT>(ids, L, p_next2, pol_idx);
        cp_async_commit();
        const int64_t tn3 = t + 3 * G;
        const uint32_t p_after = (tn3 < ntiles && node(tn3) < L.n) ? __ldg(L.vox + node(tn3)) : 0u;

        // ---- collide tile t (its values are in vcur)
        const int64_t i64 = node(t);
        double part = 0.0;
        if (i64 < L.n) {
            const int i = (int)i64;
            const M r_own = own_ref<S>(bc, L, p_cur), g = own_slope<S>(bc);
            const uint32_t seed = step_seed<S>(bc, slot);
            M d[19];
            read_vals<S, NT>(d, vcur, hi_cur, nb_cur, r_own, g);
            if (i < L.a_in) {
                const M drin = bc->inlet_mode ? M(bc->drho_in_fixed) : M(bc->drho_in[slot]);
                close_inlet(d, drin - inlet_known(d));
            } else if (i64 >= L.n - L.a_out) {
                const M uz = outlet_known(d) - M(bc->drho_out);
                close_outlet(d, uz);
            }
            collide(d, sp, sm);
            encode_node<S>(d, seed, i, [&](auto) { return r_own; }, [&](auto qc, typename S::T v) {
                constexpr int Q = decltype(qc)::value;
                P.out[Q][i] = v;
            });
            if (i64 < L.a_01) part = next_inlet_part<S>(d, L, p_cur, i, r_own, seed);
        }
        if (t < nt01) {  // tile holds plane z = 0 / z = 1 nodes (block-uniform)
            const double b = block_sum<NT>(part, sh);
            if (threadIdx.x == 0) {
                partials[t] = b;
                __threadfence();
                last = atomicAdd(counter, 1u) == (unsigned)nt01 - 1;
            }
            __syncthreads();
            if (last) {
                __threadfence();
                double s = 0.0;
                for (int64_t j = threadIdx.x; j < nt01; j += NT) s += __ldcg(partials + j);
                s = block_sum<NT>(s, sh);
                if (threadIdx.x == 0) {
                    bc->drho_in[slot ^ 1] = (bc->Q + s) / (double)L.a_in;
                    if constexpr (S::kRef) bc->sr_seed[slot ^ 1] = sr_next(bc->sr_seed[slot]);
                    *counter = 0u;
                }
            }
        }
        hi_cur = hi_next;
        nb_cur = nb_next;
        p_cur = p_next;
        p_next = p_next2;
        p_next2 = p_after;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------- monitors ---
template <class S>
__global__ void __launch_bounds__(kReduceBlock)
k_monitors(const typename S::T* __restrict__ f, DevLattice L, const BcState* bc,
           double* __restrict__ partials, unsigned* __restrict__ counter, MonitorOut* out) {
    using M = typename S::M;
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i64 = (int64_t)blockIdx.x * kReduceBlock + threadIdx.x;
    M v[5] = {M(0), M(0), M(0), M(0), M(0)};
    if (i64 < L.n) {
        const int i = (int)i64;
        const M r_own = own_ref<S>(bc, L, L.vox[i]);
        M d[19];
        for_q(AllQ{}, [&](auto qc) {
            constexpr int Q = decltype(qc)::value;
            d[Q] = S::template dec<Q>(f[(int64_t)Q * L.ns + i], r_own);
        });
        M drho, jx, jy, jz;
        moments(d, drho, jx, jy, jz);
        const M u2 = jx * jx + jy * jy + jz * jz;
        const bool bad = !isfinite((double)drho) || !isfinite((double)u2);
        v[0] = bad ? M(0) : drho;
        if (i64 < L.a_in && !bad) v[1] = jz;
        if (i64 >= L.n - L.a_out && !bad) v[2] = jz;
        v[3] = bad ? M(0) : u2;
        v[4] = bad ? M(1) : M(0);
    }
    const int nb = gridDim.x;
    double r[5];
    r[0] = block_sum_m<kReduceBlock>(v[0], sh);
    r[1] = block_sum_m<kReduceBlock>(v[1], sh);
    r[2] = block_sum_m<kReduceBlock>(v[2], sh);
    r[3] = block_max_m<kReduceBlock>(v[3], sh);
    r[4] = block_sum_m<kReduceBlock>(v[4], sh);
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

// ------------------------------------------------- steady residual ---
// Section 3.1 stopping criterion: sum_x |u(x,t) - u(x,t_ref)| and sum_x |u(x,t)|
// (|.| the Euclidean norm per node), FP64; u_ref <- u(t) for the next call.
template <class S>
__global__ void __launch_bounds__(kReduceBlock)
k_velocity_change(const typename S::T* __restrict__ f, DevLattice L, const BcState* bc,
                  double* __restrict__ u_ref,
                  double* __restrict__ partials, unsigned* __restrict__ counter, MonitorOut* out) {
    using M = typename S::M;
    __shared__ double sh[32];
    __shared__ bool last;
    const int64_t i64 = (int64_t)blockIdx.x * kReduceBlock + threadIdx.x;
    M dn = M(0), un = M(0);
    if (i64 < L.n) {
        const M r_own = own_ref<S>(bc, L, L.vox[i64]);
        M d[19];
        for_q(AllQ{}, [&](auto qc) {
            constexpr int Q = decltype(qc)::value;
            d[Q] = S::template dec<Q>(f[(int64_t)Q * L.ns + i64], r_own);
        });
        M drho, jx, jy, jz;
        moments(d, drho, jx, jy, jz);
        const M u[3] = {jx, jy, jz};
        M d2 = M(0), u2 = M(0);
        for (int c = 0; c < 3; ++c) {
            const M r = (M)u_ref[(int64_t)c * L.n + i64];
            d2 += (u[c] - r) * (u[c] - r);
            u2 += u[c] * u[c];
            u_ref[(int64_t)c * L.n + i64] = (double)u[c];
        }
        dn = sqrt(d2);
        un = sqrt(u2);
    }
    const int nb = gridDim.x;
    const double b0 = block_sum_m<kReduceBlock>(dn, sh);
    const double b1 = block_sum_m<kReduceBlock>(un, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b0;
        partials[(int64_t)nb + blockIdx.x] = b1;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a0 = 0.0, a1 = 0.0;
    for (int j = threadIdx.x; j < nb; j += kReduceBlock) {
        a0 += __ldcg(partials + j);
        a1 += __ldcg(partials + (int64_t)nb + j);
    }
    const double t0 = block_sum<kReduceBlock>(a0, sh);
    const double t1 = block_sum<kReduceBlock>(a1, sh);
    if (threadIdx.x == 0) {
        out->drho_sum = t0;  // sum |u - u_ref|
        out->q_in = t1;      // sum |u|
        *counter = 0u;
    }
}

// ---------------------------------------------------------- re-encode ---
// 16-bit formats: move the reference profile to r(z) = r0 + g z with r0 = the
// inlet density of the next step (drho_in[slot]) and g from there to the
// outlet density, re-encoding every stored value in place (each node owns its
// values).  Reads profile slot e, writes slot e ^ 1 and selects it.
template <class S>
__global__ void k_reencode(typename S::T* __restrict__ f, DevLattice L, BcState* bc, int e, int slot) {
    using M = typename S::M;
    const float r0n = (float)bc->drho_in[slot];
    const float gn = (float)((bc->drho_out - bc->drho_in[slot]) / (double)(L.nz - 1));
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        bc->ref_r0[e ^ 1] = r0n;
        bc->ref_g[e ^ 1] = gn;
        bc->ref_cur = e ^ 1;
    }
    if (i >= L.n) return;
    const int z = plane_of((uint64_t)L.vox[i], L.sz_magic);
    const M r_old = M(bc->ref_r0[e]) + M(bc->ref_g[e]) * M(z);
    const M r_new = M(r0n) + M(gn) * M(z);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        typename S::T* a = f + (int64_t)Q * L.ns + i;
        *a = S::template enc<Q>(S::template dec<Q>(*a, r_old), r_new);
    });
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
__global__ void k_export(const typename S::T* __restrict__ f, DevLattice L, const BcState* bc, O* rho,
                         O* ux, O* uy, O* uz) {
    using M = typename S::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const M r_own = own_ref<S>(bc, L, L.vox[i]);
    M d[19];
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[Q] = S::template dec<Q>(f[(int64_t)Q * L.ns + i], r_own);
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
__global__ void k_init_eq(typename S::T* __restrict__ f, DevLattice L, const BcState* bc, const double* rho,
                          const double* ux, const double* uy, const double* uz) {
    using M = typename S::M;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const M r_own = own_ref<S>(bc, L, L.vox[i]);
    const M dr = rho ? M(rho[i] - 1.0) : M(0);
    const M u[3] = {ux ? M(ux[i]) : M(0), uy ? M(uy[i]) : M(0), uz ? M(uz[i]) : M(0)};
    const M uu15 = M(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        const M xu = M(cx(Q)) * u[0] + M(cy(Q)) * u[1] + M(cz(Q)) * u[2];
        const M dq = M(wq(Q)) * (dr + M(3) * xu + M(4.5) * xu * xu - uu15);
        f[(int64_t)Q * L.ns + i] = S::template enc<Q>(dq, r_own);
    });
}

template <class S>
__global__ void k_encode(typename S::T* __restrict__ f, DevLattice L, const BcState* bc,
                         const double* __restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const typename S::M r_own = own_ref<S>(bc, L, L.vox[i]);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        f[(int64_t)Q * L.ns + i] = S::template enc<Q>((typename S::M)d[(int64_t)Q * L.n + i], r_own);
    });
}

template <class S>
__global__ void k_decode(const typename S::T* __restrict__ f, DevLattice L, const BcState* bc,
                         double* __restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.n) return;
    const typename S::M r_own = own_ref<S>(bc, L, L.vox[i]);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[(int64_t)Q * L.n + i] = (double)S::template dec<Q>(f[(int64_t)Q * L.ns + i], r_own);
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
int step_reduce_blocks(const DevLattice& L) { return (int)blocks_for(L.a_01, kBlock); }
int monitor_blocks(const DevLattice& L) { return (int)blocks_for(L.n, kReduceBlock); }

cudaError_t launch_inlet_reduce(int prec, const void* fin, int slot, const DevLattice& L, BcState* bc,
                                double* partials, unsigned* counter, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_inlet_reduce<S><<<inlet_reduce_blocks(L), kReduceBlock, 0, st>>>(
            (const typename S::T*)fin, slot, L, bc, partials, counter);
        return cudaGetLastError();
    });
}

cudaError_t launch_step(int prec, const void* fin, void* fout, int slot, const DevLattice& L, Relax r,
                        BcState* bc, double* partials, unsigned* counter, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        using M = typename S::M;
        using T = typename S::T;
        StepPtrs<T> P;
        for (int q = 0; q < 19; ++q) {
            P.in[q] = (const T*)fin + (int64_t)q * L.ns;
            P.out[q] = (T*)fout + (int64_t)q * L.ns;
        }
        // GB300_LBM_STEP_ADDR64 forces the 64-bit form (tests)
        if (19 * (uint64_t)L.ns <= 0xFFFFFFFFull && !std::getenv("GB300_LBM_STEP_ADDR64"))
            k_step<S, true><<<blocks_for(L.n, kBlock), kBlock, 0, st>>>(P, slot, L, (M)r.sp, (M)r.sm, bc,
                                                                         partials, counter);
        else
            k_step<S><<<blocks_for(L.n, kBlock), kBlock, 0, st>>>(P, slot, L, (M)r.sp, (M)r.sm, bc, partials,
                                                                   counter);
        return cudaGetLastError();
    });
}

template <class S, int NT>
cudaError_t launch_async_t(const void* fin, void* fout, int slot, const DevLattice& L, Relax r, BcState* bc,
                           double* partials, unsigned* counter, cudaStream_t st, int grid) {
    using T = typename S::T;
    using M = typename S::M;
    StepPtrs<T> P;
    for (int q = 0; q < 19; ++q) {
        P.in[q] = (const T*)fin + (int64_t)q * L.ns;
        P.out[q] = (T*)fout + (int64_t)q * L.ns;
    }
    const size_t smem = async_smem_bytes<NT>(AsyncSlot<S>::kBytes);
    k_step_async<S, NT><<<grid, NT, smem, st>>>(P, slot, L, (M)r.sp, (M)r.sm, bc, partials, counter);
    return cudaGetLastError();
}

template <class S, int NT>
cudaError_t config_async_t(int* grid, int64_t n) {
    const size_t smem = async_smem_bytes<NT>(AsyncSlot<S>::kBytes);
    cudaError_t e = cudaFuncSetAttribute(k_step_async<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_async<S, NT>, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t ntiles = (n + NT - 1) / NT;
    *grid = (int)std::min<int64_t>((int64_t)per_sm * sms, ntiles);
    return cudaSuccess;
}

cudaError_t launch_monitors(int prec, const void* f, const DevLattice& L, const BcState* bc, double* partials,
                            unsigned* counter, MonitorOut* out, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_monitors<S><<<monitor_blocks(L), kReduceBlock, 0, st>>>((const typename S::T*)f, L, bc,
                                                                   partials, counter, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_velocity_change(int prec, const void* f, const DevLattice& L, const BcState* bc, double* u_ref,
                                   double* partials, unsigned* counter, MonitorOut* out, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_velocity_change<S><<<monitor_blocks(L), kReduceBlock, 0, st>>>((const typename S::T*)f, L, bc, u_ref,
                                                                         partials, counter, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_reencode(int prec, void* f, const DevLattice& L, BcState* bc, int e, int slot,
                            cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        if constexpr (S::kRef) {
            k_reencode<S><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L, bc, e, slot);
            return cudaGetLastError();
        } else {
            return cudaSuccess;
        }
    });
}

cudaError_t launch_export(int prec, const void* f, const DevLattice& L, const BcState* bc, void* rho, void* ux,
                          void* uy, void* uz, int out_double, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        if (out_double)
            k_export<S, double><<<blocks_for(L.n, 256), 256, 0, st>>>(
                (const typename S::T*)f, L, bc, (double*)rho, (double*)ux, (double*)uy, (double*)uz);
        else
            k_export<S, float><<<blocks_for(L.n, 256), 256, 0, st>>>(
                (const typename S::T*)f, L, bc, (float*)rho, (float*)ux, (float*)uy, (float*)uz);
        return cudaGetLastError();
    });
}

cudaError_t launch_init_eq(int prec, void* f, const DevLattice& L, const BcState* bc, const double* rho,
                           const double* ux, const double* uy, const double* uz, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_init_eq<S><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L, bc, rho, ux, uy, uz);
        return cudaGetLastError();
    });
}

cudaError_t launch_encode(int prec, void* f, const DevLattice& L, const BcState* bc, const double* d,
                          cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_encode<S><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L, bc, d);
        return cudaGetLastError();
    });
}

cudaError_t launch_decode(int prec, const void* f, const DevLattice& L, const BcState* bc, double* d,
                          cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_decode<S><<<blocks_for(L.n, 256), 256, 0, st>>>((const typename S::T*)f, L, bc, d);
        return cudaGetLastError();
    });
}

cudaError_t launch_aa_step(int prec, void* f, int odd, int slot, const DevLattice& L, Relax r, BcState* bc,
                           double* partials, unsigned* counter, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        using M = typename S::M;
        {
            AAPtrs<typename S::T> F;
            for (int q = 0; q < 19; ++q) F.row[q] = (typename S::T*)f + (int64_t)q * L.ns;
            // every element offset of the buffer fits in 32 bits; the environment
            // variable GB300_LBM_AA_ADDR64 forces the 64-bit form (for tests)
            const bool off32 = 19 * (uint64_t)L.ns <= 0xFFFFFFFFull && !std::getenv("GB300_LBM_AA_ADDR64");
            if (odd && off32)
                k_step_aa<S, true, true><<<blocks_for(L.n, kBlock), kBlock, 0, st>>>(
                    F, slot, L, (M)r.sp, (M)r.sm, bc, partials, counter);
            else if (odd)
                k_step_aa<S, true><<<blocks_for(L.n, kBlock), kBlock, 0, st>>>(F, slot, L, (M)r.sp, (M)r.sm, bc,
                                                                                partials, counter);
            else
                k_step_aa<S, false><<<blocks_for(L.n, kBlock), kBlock, 0, st>>>(F, slot, L, (M)r.sp, (M)r.sm, bc,
                                                                                 partials, counter);
            return cudaGetLastError();
        }
    });
}

cudaError_t launch_aa_swap(int prec, void* f, const DevLattice& L, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_aa_swap<typename S::T><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L.n, L.ns);
        return cudaGetLastError();
    });
}

cudaError_t launch_aa_unstream(int prec, void* f, const DevLattice& L, const BcState* bc, cudaStream_t st) {
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        k_aa_unstream<S><<<blocks_for(L.n, 256), 256, 0, st>>>((typename S::T*)f, L, bc);
        return cudaGetLastError();
    });
}

cudaError_t configure_step(int prec, int variant, const DevLattice& L, StepConfig* cfg) {
    cfg->variant = variant;
    cfg->grid = 0;
    if (variant == 0) return cudaSuccess;
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        if (variant == 1) return config_async_t<S, 256>(&cfg->grid, L.n);
        if (variant == 2) return config_async_t<S, 128>(&cfg->grid, L.n);
        return cudaErrorInvalidValue;
    });
}

cudaError_t launch_step_cfg(int prec, const StepConfig& cfg, const void* fin, void* fout, int slot,
                            const DevLattice& L, Relax r, BcState* bc, double* partials, unsigned* counter,
                            cudaStream_t st) {
    if (cfg.variant == 0) return launch_step(prec, fin, fout, slot, L, r, bc, partials, counter, st);
    return dispatch(prec, [&](auto s) {
        using S = decltype(s);
        if (cfg.variant == 1)
            return launch_async_t<S, 256>(fin, fout, slot, L, r, bc, partials, counter, st, cfg.grid);
        if (cfg.variant == 2)
            return launch_async_t<S, 128>(fin, fout, slot, L, r, bc, partials, counter, st, cfg.grid);
        return cudaErrorInvalidValue;
    });
}

}  // namespace lbm
