// Batched ensemble: many independent porous sub-volumes of uneven size, each
// with its own flux target, advanced by ONE kernel launch per time step.
//
// All members share one structure-of-arrays distribution store.  Each member's
// pore list (z, y, x order, inlet plane first, outlet plane last) starts on a
// 256-node tile boundary, its padded id grid holds global pore indices, and a
// per-tile member table routes every block to its member's parameters.  The
// step is the single-lattice step (pull with halfway bounce-back, Appendix B
// closures with the inlet density of Eq. potential, collision, store) with the
// member's own boundary scalars; the next step's inlet density of every member
// is formed in the same launch (FP64, deterministic last-tile finish per
// member).  Two launch forms: one launch per step, runs of 64 steps replaying a
// captured CUDA graph; or one persistent cooperative launch for all steps of a
// call, with a bounded grid barrier between steps.  Each form comes with two
// register caps; lbm_batch_autotune times the four on the ensemble and keeps
// the fastest.
#include <cuda_runtime.h>

#include <algorithm>
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

constexpr int kTile = 256;
constexpr int kBatchGraphSteps = 64;
constexpr int64_t kBatchReencodeInterval = 1024;

// Per-member parameters and boundary state (device, mutable).
struct Member {
    int64_t base;       // first global pore slot (multiple of kTile)
    int64_t n;          // pore nodes
    int64_t a_in;       // inlet pore nodes: local [0, a_in)
    int64_t a_out;      // outlet pore nodes: local [n - a_out, n)
    int64_t a_01;       // pore nodes on planes z = 0, 1: local [0, a_01)
    int64_t grid_base;  // first padded voxel of the member's id grid
    uint64_t sz_magic;  // ceil(2^64 / ((nx+2)(ny+2)))
    int nz;
    int goff[19];       // padded-grid offsets of the pull sources
    double Q;           // prescribed inlet flux
    double drho_out;    // outlet density - 1
    double drho_in[2];  // inlet density - 1 for the step reading buffer c
    float ref_r0[2], ref_g[2];  // 16-bit reference profile slots
    int ref_cur;
    uint32_t sr_seed[2];        // stochastic-rounding seed of the step reading buffer c (16-bit)
};

// LBM_BATCH16_PAIR_SCATTER: as LBM_AA16_PAIR_SCATTER, for the ensemble's
// gather-scatter step.  Measured on the 64-pack FP16-dev ensemble, the
// opposite order from the single lattice: its AA step takes 1.234 ms with one
// conversion per pair and 1.243 ms with one per value.
#ifndef LBM_BATCH16_PAIR_SCATTER
#define LBM_BATCH16_PAIR_SCATTER 1
#endif

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
        r = lane < kTile / 32 ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

template <class S>
__device__ __forceinline__ typename S::M member_ref(const Member& m, int64_t p_global) {
    using M = typename S::M;
    if constexpr (S::kRef) {
        const int z = plane_of((uint64_t)(p_global - m.grid_base), m.sz_magic);
        const int c = m.ref_cur;
        return M(m.ref_r0[c]) + M(m.ref_g[c]) * M(z);
    } else {
        return M(0);
    }
}
template <class S>
__device__ __forceinline__ typename S::M member_slope(const Member& m) {
    using M = typename S::M;
    if constexpr (S::kRef) return M(m.ref_g[m.ref_cur]);
    else return M(0);
}

// Loads of values that other blocks of the same launch may have written (the
// persistent launch: distributions and member scalars of the previous step) go
// through L2 (ld.global.cg); per-step launches use ordinary loads.
template <bool COH, class T>
__device__ __forceinline__ T ld_state(const T* p) {
    if constexpr (!COH) {
        return *p;
    } else if constexpr (sizeof(T) == 2) {
        const unsigned short u = __ldcg(reinterpret_cast<const unsigned short*>(p));
        T v;
        memcpy(&v, &u, 2);
        return v;
    } else {
        return __ldcg(p);
    }
}

// OFF32 (per-step launches, ensembles of 19 ns < 2^32 elements): the source is
// fin plus one 32-bit element offset, its row chosen by a 32-bit select, rather
// than one of two 64-bit addresses.  Measured on the 64-pack FP16-dev ensemble:
// the step 0.981 against 1.141 ms (48-register cap), and no spills at that cap.
template <class S, int Q, bool COH = false, bool OFF32 = false>
__device__ __forceinline__ typename S::M pull_b(const typename S::T* fin, int64_t ns,
                                                const int* __restrict__ grid, const Member& m,
                                                int64_t p, int64_t i, typename S::M r_own,
                                                typename S::M g) {
    using M = typename S::M;
    if (Q == 0) return S::template dec<0>(ld_state<COH>(fin + i), r_own);
    const int id = __ldg(grid + p + m.goff[Q]);
    if constexpr (OFF32) {
        const bool pore = id >= 0;
        const uint32_t off =
            pore ? (uint32_t)Q * (uint32_t)ns + (uint32_t)id : (uint32_t)opp(Q) * (uint32_t)ns + (uint32_t)i;
        return S::template dec<Q>(ld_state<COH>(fin + off), pore ? r_own - M(cz(Q)) * g : r_own);
    } else {
        if (id >= 0) return S::template dec<Q>(ld_state<COH>(fin + (int64_t)Q * ns + id), r_own - M(cz(Q)) * g);
        return S::template dec<Q>(ld_state<COH>(fin + (int64_t)opp(Q) * ns + i), r_own);
    }
}

// Same contribution rule as the single-lattice step (see lbm_kernels.cu).
template <class S>
__device__ __forceinline__ double next_inlet_part_b(const typename S::M* d, const int* __restrict__ grid,
                                                    const Member& m, int64_t p, int64_t il,
                                                    typename S::M r_own, uint32_t seed, int64_t i) {
    double s = 0.0;
    auto val = [&](auto qc) -> double {
        constexpr int Q = decltype(qc)::value;
        return (double)S::template dec<Q>(S::template enc_sr<Q>(d[Q], r_own, sr_key<S>(seed, i, Q)), r_own);
    };
    auto dest_is_pore = [&](auto qc) -> bool {
        constexpr int Q = decltype(qc)::value;
        return __ldg(grid + p + m.goff[opp(Q)]) >= 0;
    };
    if (il < m.a_in) {
        for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 7, 8, 9, 10>{}, [&](auto qc) { s += val(qc); });
        for_q(std::integer_sequence<int, 5, 11, 14, 15, 18>{},
              [&](auto qc) { if (!dest_is_pore(qc)) s += 2.0 * val(qc); });
    } else {
        for_q(std::integer_sequence<int, 6, 12, 13, 16, 17>{},
              [&](auto qc) { if (dest_is_pore(qc)) s += 2.0 * val(qc); });
    }
    return s;
}

// Per-member reduction of `part` over the member's tiles [0, ntiles_member):
// partials per global tile, a ticket per member, the last tile writes.
template <class F>
__device__ __forceinline__ void member_reduce(double part, int64_t tile, int64_t tile0, int64_t ntm,
                                              double* partials, unsigned* counter, double* sh, F&& finish) {
    __shared__ bool last;
    const double b = block_sum(part, sh);
    if (threadIdx.x == 0) {
        partials[tile] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)ntm - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < ntm; j += kTile) s += __ldcg(partials + tile0 + j);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) {
            finish(s);
            *counter = 0u;
        }
    }
}

// One 256-node tile of one step: the single-lattice step with the member's own
// boundary scalars, and the member's next inlet density (last tile finishes).
template <class S, bool COH, bool OFF32 = false>
__device__ __forceinline__ void batch_tile_step(const typename S::T* fin, typename S::T* fout, int64_t ns, int slot,
                                                int64_t tile, const uint32_t* __restrict__ vox,
                                                const int* __restrict__ grid, const int* __restrict__ tile_member,
                                                Member* members, typename S::M sp, typename S::M sm,
                                                double* partials, unsigned* counters, double* sh) {
    using M = typename S::M;
    const int mi = tile_member[tile];
    const Member& m = members[mi];
    const int64_t tile0 = m.base / kTile;
    const int64_t i = tile * kTile + threadIdx.x;
    const int64_t il = i - m.base;
    double part = 0.0;
    if (il < m.n) {
        const int64_t p = vox[i];
        const M r_own = member_ref<S>(m, p), g = member_slope<S>(m);
        const uint32_t seed = S::kRef ? ld_state<COH>(&m.sr_seed[slot]) : 0u;
        M d[19];
        for_q(AllQ{}, [&](auto qc) {
            constexpr int Q = decltype(qc)::value;
            d[Q] = pull_b<S, Q, COH, OFF32>(fin, ns, grid, m, p, i, r_own, g);
        });
        if (il < m.a_in) {
            close_inlet(d, M(ld_state<COH>(&m.drho_in[slot])) - inlet_known(d));
        } else if (il >= m.n - m.a_out) {
            close_outlet(d, outlet_known(d) - M(m.drho_out));
        }
        collide(d, sp, sm);
        encode_node<S>(d, seed, i, [&](auto) { return r_own; }, [&](auto qc, typename S::T v) {
            constexpr int Q = decltype(qc)::value;
            fout[(int64_t)Q * ns + i] = v;
        });
        if (il < m.a_01) part = next_inlet_part_b<S>(d, grid, m, p, il, r_own, seed, i);
    }
    const int64_t nt01 = (m.a_01 + kTile - 1) / kTile;
    if (tile - tile0 < nt01)
        member_reduce(part, tile, tile0, nt01, partials, counters + mi, sh, [&](double s) {
            members[mi].drho_in[slot ^ 1] = (m.Q + s) / (double)m.a_in;
            if constexpr (S::kRef) members[mi].sr_seed[slot ^ 1] = sr_next(ld_state<COH>(&m.sr_seed[slot]));
        });
}

// LBM_BATCH_PREFETCH: the per-step and gather-scatter AA kernels ask L2 for the
// rows of the tile that many tiles ahead (bulk prefetch, nothing waited for);
// 0 = off.  A launch covers every tile once, so gridDim.x * kTile is the padded
// slot count, which equals ns and the length of the voxel list; each range
// starts at a multiple of kTile slots.  Measured on the 64-pack FP16-dev
// ensemble: the per-step form (48-register cap) 1.332 ms per step without, 1.204
// at 32 tiles ahead, 1.190 at 224, 1.188 at 384 and 640.
#ifndef LBM_BATCH_PREFETCH
#define LBM_BATCH_PREFETCH 384
#endif
template <class T>
__device__ __forceinline__ void batch_prefetch(const T* row0, int64_t ns, const uint32_t* vox) {
    if constexpr (LBM_BATCH_PREFETCH > 0) {
        const int64_t s = ((int64_t)blockIdx.x + LBM_BATCH_PREFETCH) * kTile;
        const int64_t end = (int64_t)gridDim.x * kTile;
        const int t = (int)threadIdx.x;
        if (t < 19) l2_prefetch_range(row0 + (int64_t)t * ns, s, kTile, end);
        else if (t == 19) l2_prefetch_range(vox, s, kTile, end);
    }
}

// Resident blocks per SM a configuration compiles for (register cap); FP64 is
// left unconstrained.
template <class S, int MINB>
constexpr int batch_min_blocks() {
    return sizeof(typename S::M) == 8 ? 1 : MINB;
}

// One step, one tile per block.
template <class S, int MINB, bool OFF32 = false>
__global__ void __launch_bounds__(kTile, batch_min_blocks<S, MINB>())
k_batch_step(const typename S::T* __restrict__ fin, typename S::T* __restrict__ fout, int64_t ns, int slot,
             const uint32_t* __restrict__ vox, const int* __restrict__ grid, const int* __restrict__ tile_member,
             Member* members, typename S::M sp, typename S::M sm, double* __restrict__ partials,
             unsigned* __restrict__ counters) {
    __shared__ double sh[32];
    batch_prefetch(fin, ns, vox);
    batch_tile_step<S, false, OFF32>(fin, fout, ns, slot, blockIdx.x, vox, grid, tile_member, members, sp, sm,
                                     partials, counters, sh);
}

// Grid barrier of the persistent launch.  Thread 0 of every block arrives on a
// counter; the last arrival resets it and advances the generation, the others
// wait for the generation to change.  The wait is bounded: after `limit` SM
// cycles the block records a timeout and the caller returns, so a block that
// never arrives cannot hang the GPU.
struct GridBarrier {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned nblocks, unsigned& gen, long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = gen;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicExch(&bar->gen, g + 1u);
            ok = 1;
        } else {
            ok = 0;
            const long long t0 = clock64();
            while (true) {
                if (*(volatile unsigned*)&bar->gen != g) {
                    ok = 1;
                    break;
                }
                if (clock64() - t0 > limit) break;
                __nanosleep(64);
            }
            if (!ok) atomicExch(&bar->err, 1);
        }
        __threadfence();
        gen = g + 1u;
    }
    __syncthreads();
    return ok != 0;
}

// `nsteps` steps in one cooperative launch: blocks walk the tiles with a grid
// stride, a bounded grid barrier separates the steps.  Step s reads buffer
// slot0 ^ (s & 1).
template <class S, int MINB>
__global__ void __launch_bounds__(kTile, batch_min_blocks<S, MINB>())
k_batch_persistent(typename S::T* f0, typename S::T* f1, int64_t ns, int slot0, int nsteps, int64_t ntiles,
                   const uint32_t* __restrict__ vox, const int* __restrict__ grid,
                   const int* __restrict__ tile_member, Member* members, typename S::M sp, typename S::M sm,
                   double* partials, unsigned* counters, GridBarrier* bar, long long limit) {
    __shared__ double sh[32];
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = *(volatile unsigned*)&bar->gen;
    for (int s = 0; s < nsteps; ++s) {
        const int slot = slot0 ^ (s & 1);
        const typename S::T* fin = slot ? f1 : f0;
        typename S::T* fout = slot ? f0 : f1;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
            batch_tile_step<S, true>(fin, fout, ns, slot, tile, vox, grid, tile_member, members, sp, sm, partials,
                                     counters, sh);
        if (!grid_barrier(bar, gridDim.x, gen, limit)) return;
    }
}

// Barrier check: `nblocks` blocks meet at a barrier that expects `expected`
// arrivals.  With expected == nblocks it completes; with more it must time out
// and set the error flag.
__global__ void k_barrier_probe(GridBarrier* bar, unsigned expected, long long limit) {
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = *(volatile unsigned*)&bar->gen;
    grid_barrier(bar, expected, gen, limit);
}

// ----------------------------------------------------- AA pattern (batch) ---
// The single-lattice AA pattern (see lbm_kernels.cu) on the shared store: the
// state rests in the pull layout between calls; a call swaps every node's
// opposite pairs, alternates gather-scatter (odd) and node-local (even) steps,
// and swaps back (after an odd count an un-stream swap comes first).  Ids are
// global pore indices, so the scatter stays inside the member.  16-bit values
// are encoded with the reference of the plane of the node that holds them.  In
// the 32-bit offset form the gather-scatter step stages each direction's gather
// offset in shared memory (LBM_BATCH_AA_STAGE): the scatter destination of q is
// the slot the gather of opp(q) read, so the scatter needs neither the voxel
// index nor the ids again; otherwise it loads them again for the scatter.
// Row pointers of the store as kernel parameters (constant bank): no registers
// spent on 19 row addresses.
template <class T>
struct Rows {
    T* row[19];
};

// Measured on the 64-member FP16-dev ensemble (same-call A/B, bitwise equal
// states): AA configuration 1.157 -> 1.068 ms per step, AA-capped 1.223 -> 1.136.
#ifndef LBM_BATCH_AA_STAGE
#define LBM_BATCH_AA_STAGE 1
#endif

template <class S, bool ODD, int MINB, bool OFF32 = false>
__global__ void __launch_bounds__(kTile, batch_min_blocks<S, MINB>())
k_batch_aa(const Rows<typename S::T> F, int slot, const uint32_t* __restrict__ vox,
           const int* __restrict__ grid, const int* __restrict__ tile_member, Member* members, typename S::M sp,
           typename S::M sm, double* __restrict__ partials, unsigned* __restrict__ counters) {
    using M = typename S::M;
    __shared__ double sh[32];
    constexpr bool kStage = ODD && OFF32 && LBM_BATCH_AA_STAGE;
    __shared__ uint32_t soff[kStage ? 18 : 1][kStage ? kTile : 1];  // gather offset per direction and node
    if constexpr (ODD) batch_prefetch(F.row[0], F.row[1] - F.row[0], vox);  // rows are ns apart, as launched
    const int64_t tile = blockIdx.x;
    const int mi = tile_member[tile];
    const Member& m = members[mi];
    const int64_t tile0 = m.base / kTile;
    const int64_t i = tile * kTile + threadIdx.x;
    const int64_t il = i - m.base;
    double part = 0.0;
    if (il < m.n) {
        const int64_t p = vox[i];
        const M r_own = member_ref<S>(m, p), g = member_slope<S>(m);
        const uint32_t seed = S::kRef ? m.sr_seed[slot] : 0u;
        M d[19];
        if constexpr (ODD) {
            d[0] = S::template dec<0>(F.row[0][i], r_own);
            const uint32_t ns32 = (uint32_t)(F.row[1] - F.row[0]);  // rows are ns apart, as launched
            for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value + 1;
                const int id = __ldg(grid + p + m.goff[Q]);
                if constexpr (OFF32) {
                    const bool pore = id >= 0;
                    const uint32_t off = pore ? (uint32_t)opp(Q) * ns32 + (uint32_t)id : (uint32_t)Q * ns32 + (uint32_t)i;
                    if constexpr (kStage) soff[Q - 1][threadIdx.x] = off;
                    d[Q] = S::template dec<Q>(F.row[0][off], pore ? r_own - M(cz(Q)) * g : r_own);
                } else {
                    d[Q] = id >= 0 ? S::template dec<Q>(F.row[opp(Q)][id], r_own - M(cz(Q)) * g)
                                   : S::template dec<Q>(F.row[Q][i], r_own);
                }
            });
        } else if constexpr (OFF32) {
            const uint32_t ns32 = (uint32_t)(F.row[1] - F.row[0]);
            for_q(AllQ{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value;
                d[Q] = S::template dec<Q>(F.row[0][(uint32_t)Q * ns32 + (uint32_t)i], r_own);
            });
        } else {
            for_q(AllQ{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value;
                d[Q] = S::template dec<Q>(F.row[Q][i], r_own);
            });
        }
        if (il < m.a_in) {
            close_inlet(d, M(m.drho_in[slot]) - inlet_known(d));
        } else if (il >= m.n - m.a_out) {
            close_outlet(d, outlet_known(d) - M(m.drho_out));
        }
        collide(d, sp, sm);
        // an opaque copy of the node index for the stores (sharing the load
        // addresses would keep 19 64-bit addresses live across the collision)
        int64_t j;
        asm volatile("mov.b64 %0, %1;" : "=l"(j) : "l"(i));
        if constexpr (kStage) {
            F.row[0][j] = S::template enc_sr<0>(d[0], r_own, sr_key<S>(seed, i, 0));
            // the destination of Q is the gather source of opp(Q): row Q for a pore
            // there, row opp(Q) (bounce-back) otherwise
            const uint32_t ns32 = (uint32_t)(F.row[1] - F.row[0]);
            for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                constexpr int Q = decltype(qc)::value + 1;
                const uint32_t off = soff[opp(Q) - 1][threadIdx.x];
                M r = r_own;
                if constexpr (S::kRef && cz(Q) != 0) {
                    const bool pore = (Q & 1) ? off < (uint32_t)(Q + 1) * ns32 : off >= (uint32_t)Q * ns32;
                    r = pore ? r_own + M(cz(Q)) * g : r_own;
                }
                F.row[0][off] = S::template enc_sr<Q>(d[Q], r, sr_key<S>(seed, i, Q));
            });
        } else if constexpr (ODD) {
            const int64_t ps = __ldg(vox + j);
            F.row[0][j] = S::template enc_sr<0>(d[0], r_own, sr_key<S>(seed, i, 0));
            if constexpr (OFF32) {
                // one store per value at row 0 plus a 32-bit offset, destination row and plane selected
                const uint32_t ns32 = (uint32_t)(F.row[1] - F.row[0]);
                for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                    constexpr int Q = decltype(qc)::value + 1;
                    const int dst = __ldg(grid + ps + m.goff[opp(Q)]);  // x + xi_Q is the pull source of opp(Q)
                    const bool pore = dst >= 0;
                    F.row[0][pore ? (uint32_t)Q * ns32 + (uint32_t)dst : (uint32_t)opp(Q) * ns32 + (uint32_t)j] =
                        S::template enc_sr<Q>(d[Q], pore ? r_own + M(cz(Q)) * g : r_own, sr_key<S>(seed, i, Q));
                });
            } else if constexpr (S::kRef && !LBM_BATCH16_PAIR_SCATTER) {
                for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                    constexpr int Q = decltype(qc)::value + 1;
                    const int dst = __ldg(grid + ps + m.goff[opp(Q)]);  // x + xi_Q is the pull source of opp(Q)
                    const uint32_t key = sr_key<S>(seed, i, Q);
                    if (dst >= 0) F.row[Q][dst] = S::template enc_sr<Q>(d[Q], r_own + M(cz(Q)) * g, key);
                    else F.row[opp(Q)][j] = S::template enc_sr<Q>(d[Q], r_own, key);
                });
            } else if constexpr (S::kRef) {
                // per opposite pair one stochastic conversion, then one store per value
                for_q(std::make_integer_sequence<int, 9>{}, [&](auto pc) {
                    constexpr int Q = 2 * decltype(pc)::value + 1;
                    const int dq = __ldg(grid + ps + m.goff[Q + 1]);   // x + xi_Q is the pull source of Q + 1
                    const int dq1 = __ldg(grid + ps + m.goff[Q]);      // and x - xi_Q that of Q
                    const uint32_t h = S::template enc_sr2<Q>(d[Q], dq >= 0 ? r_own + M(cz(Q)) * g : r_own, d[Q + 1],
                                                              dq1 >= 0 ? r_own - M(cz(Q)) * g : r_own,
                                                              sr_key<S>(seed, i, Q), sr_key<S>(seed, i, Q + 1));
                    if (dq >= 0) F.row[Q][dq] = S::half_of(h, true);
                    else F.row[Q + 1][j] = S::half_of(h, true);
                    if (dq1 >= 0) F.row[Q + 1][dq1] = S::half_of(h, false);
                    else F.row[Q][j] = S::half_of(h, false);
                });
            } else {
                for_q(std::make_integer_sequence<int, 18>{}, [&](auto qc) {
                    constexpr int Q = decltype(qc)::value + 1;
                    const int dst = __ldg(grid + ps + m.goff[opp(Q)]);  // x + xi_Q is the pull source of opp(Q)
                    if (dst >= 0) F.row[Q][dst] = d[Q];
                    else F.row[opp(Q)][j] = d[Q];
                });
            }
        } else if constexpr (OFF32) {
            const uint32_t ns32 = (uint32_t)(F.row[1] - F.row[0]);
            encode_node<S>(d, seed, i, [&](auto) { return r_own; }, [&](auto qc, typename S::T v) {
                constexpr int Q = decltype(qc)::value;
                F.row[0][(uint32_t)opp(Q) * ns32 + (uint32_t)j] = v;
            });
        } else {
            encode_node<S>(d, seed, i, [&](auto) { return r_own; }, [&](auto qc, typename S::T v) {
                constexpr int Q = decltype(qc)::value;
                F.row[opp(Q)][j] = v;
            });
        }
        if (il < m.a_01) {
            // the counted values land on plane 0 (odd step: from plane 1 encoded with plane 0's reference)
            auto val = [&](auto qc) -> double {
                constexpr int Q = decltype(qc)::value;
                const M rq = (ODD && cz(Q) < 0) ? r_own - g : r_own;
                return (double)S::template dec<Q>(S::template enc_sr<Q>(d[Q], rq, sr_key<S>(seed, i, Q)), rq);
            };
            auto dest_is_pore = [&](auto qc) -> bool {
                constexpr int Q = decltype(qc)::value;
                return __ldg(grid + p + m.goff[opp(Q)]) >= 0;
            };
            if (il < m.a_in) {
                for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 7, 8, 9, 10>{}, [&](auto qc) { part += val(qc); });
                for_q(std::integer_sequence<int, 5, 11, 14, 15, 18>{},
                      [&](auto qc) { if (!dest_is_pore(qc)) part += 2.0 * val(qc); });
            } else {
                for_q(std::integer_sequence<int, 6, 12, 13, 16, 17>{},
                      [&](auto qc) { if (dest_is_pore(qc)) part += 2.0 * val(qc); });
            }
        }
    }
    const int64_t nt01 = (m.a_01 + kTile - 1) / kTile;
    if (tile - tile0 < nt01)
        member_reduce(part, tile, tile0, nt01, partials, counters + mi, sh, [&](double s) {
            members[mi].drho_in[slot ^ 1] = (m.Q + s) / (double)m.a_in;
            if constexpr (S::kRef) members[mi].sr_seed[slot ^ 1] = sr_next(m.sr_seed[slot]);
        });
}

// Opposite-pair swap of every slot (padding slots included; they are never read).
template <class T>
__global__ void k_batch_aa_swap(T* __restrict__ f, int64_t total, int64_t ns) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    T v[19];
#pragma unroll
    for (int q = 1; q < 19; ++q) v[q] = f[(int64_t)q * ns + i];
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        f[(int64_t)q * ns + i] = v[q + 1];
        f[(int64_t)(q + 1) * ns + i] = v[q];
    }
}

// Layout I -> S after an odd step count (pairwise swap with the pull source,
// 16-bit values re-encoded to their new holder's plane).
template <class S>
__global__ void __launch_bounds__(kTile)
k_batch_aa_unstream(typename S::T* __restrict__ f, int64_t ns, const uint32_t* __restrict__ vox,
                    const int* __restrict__ grid, const int* __restrict__ tile_member, const Member* members) {
    using M = typename S::M;
    using T = typename S::T;
    const int64_t tile = blockIdx.x;
    const Member& m = members[tile_member[tile]];
    const int64_t i = tile * kTile + threadIdx.x;
    if (i - m.base >= m.n) return;
    const int64_t p = vox[i];
    const M r_own = member_ref<S>(m, p), g = member_slope<S>(m);
    int id[19];
    T ta[19], tb[19];
    for_q(std::integer_sequence<int, 1, 3, 5, 7, 9, 11, 13, 15, 17>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        id[Q] = __ldg(grid + p + m.goff[Q]);
    });
    for_q(std::integer_sequence<int, 1, 3, 5, 7, 9, 11, 13, 15, 17>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        if (id[Q] >= 0) {
            ta[Q] = f[(int64_t)Q * ns + i];
            tb[Q] = f[(int64_t)(Q + 1) * ns + id[Q]];
        }
    });
    for_q(std::integer_sequence<int, 1, 3, 5, 7, 9, 11, 13, 15, 17>{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        if (id[Q] >= 0) {
            if constexpr (S::kRef) {
                const M r_src = r_own - M(cz(Q)) * g;
                f[(int64_t)Q * ns + i] = S::template enc<Q>(S::template dec<Q>(tb[Q], r_src), r_own);
                f[(int64_t)(Q + 1) * ns + id[Q]] = S::template enc<Q>(S::template dec<Q>(ta[Q], r_own), r_src);
            } else {
                f[(int64_t)Q * ns + i] = tb[Q];
                f[(int64_t)(Q + 1) * ns + id[Q]] = ta[Q];
            }
        }
    });
}

// Inlet density of every member by a pull over its inlet plane (states set
// from outside a step).  Grid: all tiles; tiles past a member's inlet exit.
template <class S>
__global__ void __launch_bounds__(kTile)
k_batch_inlet(const typename S::T* __restrict__ fin, int64_t ns, int slot, const uint32_t* __restrict__ vox,
              const int* __restrict__ grid, const int* __restrict__ tile_member, Member* members,
              double* __restrict__ partials, unsigned* __restrict__ counters) {
    using M = typename S::M;
    __shared__ double sh[32];
    const int64_t tile = blockIdx.x;
    const int mi = tile_member[tile];
    const Member& m = members[mi];
    const int64_t tile0 = m.base / kTile;
    const int64_t nti = (m.a_in + kTile - 1) / kTile;
    if (tile - tile0 >= nti) return;  // block-uniform
    const int64_t i = tile * kTile + threadIdx.x;
    const int64_t il = i - m.base;
    double k = 0.0;
    if (il < m.a_in) {
        const int64_t p = vox[i];
        const M r_own = member_ref<S>(m, p), g = member_slope<S>(m);
        M d[19];
        for_q(std::integer_sequence<int, 0, 1, 2, 3, 4, 6, 7, 8, 9, 10, 12, 13, 16, 17>{}, [&](auto qc) {
            constexpr int Q = decltype(qc)::value;
            d[Q] = pull_b<S, Q>(fin, ns, grid, m, p, i, r_own, g);
        });
        k = (double)d[0] + (double)d[1] + (double)d[2] + (double)d[3] + (double)d[4] + (double)d[7] +
            (double)d[8] + (double)d[9] + (double)d[10] +
            2.0 * ((double)d[6] + (double)d[12] + (double)d[13] + (double)d[16] + (double)d[17]);
    }
    member_reduce(k, tile, tile0, nti, partials, counters + mi, sh, [&](double s) {
        members[mi].drho_in[slot] = (m.Q + s) / (double)m.a_in;
    });
}

// Sum of u_z over a member's inlet (which = 0) or outlet (which = 1) plane of
// the stored state; grid = that member's tiles.
template <class S>
__global__ void __launch_bounds__(kTile)
k_batch_face_flux(const typename S::T* __restrict__ f, int64_t ns, const uint32_t* __restrict__ vox,
                  const Member* members, int mi, int which, double* __restrict__ partials,
                  unsigned* __restrict__ counter, double* out) {
    using M = typename S::M;
    __shared__ double sh[32];
    const Member& m = members[mi];
    const int64_t tile0 = m.base / kTile;
    const int64_t tile = tile0 + blockIdx.x;
    const int64_t i = tile * kTile + threadIdx.x;
    const int64_t il = i - m.base;
    double v = 0.0;
    const bool on = which == 0 ? il < m.a_in : (il >= m.n - m.a_out && il < m.n);
    if (on) {
        const M r_own = member_ref<S>(m, vox[i]);
        M d[19];
        for_q(AllQ{}, [&](auto qc) {
            constexpr int Q = decltype(qc)::value;
            d[Q] = S::template dec<Q>(f[(int64_t)Q * ns + i], r_own);
        });
        M drho, jx, jy, jz;
        moments(d, drho, jx, jy, jz);
        v = (double)jz;
    }
    member_reduce(v, tile, tile0, (int64_t)gridDim.x, partials, counter, sh, [&](double s) { *out = s; });
}

template <class S>
__global__ void k_batch_reencode(typename S::T* __restrict__ f, int64_t ns, const uint32_t* __restrict__ vox,
                                 const int* __restrict__ tile_member, Member* members, int e, int slot,
                                 int64_t total) {
    using M = typename S::M;
    const int64_t i = (int64_t)blockIdx.x * kTile + threadIdx.x;
    if (i >= total) return;
    const int mi = tile_member[blockIdx.x];
    Member& m = members[mi];
    const float r0n = (float)m.drho_in[slot];
    const float gn = (float)((m.drho_out - m.drho_in[slot]) / (double)(m.nz - 1));
    const int64_t il = i - m.base;
    if (il == 0) {
        m.ref_r0[e ^ 1] = r0n;
        m.ref_g[e ^ 1] = gn;
        m.ref_cur = e ^ 1;
    }
    if (il >= m.n) return;
    const int z = plane_of((uint64_t)(vox[i] - m.grid_base), m.sz_magic);
    const M r_old = M(m.ref_r0[e]) + M(m.ref_g[e]) * M(z);
    const M r_new = M(r0n) + M(gn) * M(z);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        typename S::T* a = f + (int64_t)Q * ns + i;
        *a = S::template enc<Q>(S::template dec<Q>(*a, r_old), r_new);
    });
}

// d = f - w for one member, pore order, row stride n (double) <-> storage.
template <class S>
__global__ void k_batch_encode(typename S::T* __restrict__ f, int64_t ns, const uint32_t* __restrict__ vox,
                               const Member* members, int mi, const double* __restrict__ d) {
    const Member& m = members[mi];
    const int64_t il = (int64_t)blockIdx.x * kTile + threadIdx.x;
    if (il >= m.n) return;
    const int64_t i = m.base + il;
    const typename S::M r_own = member_ref<S>(m, vox[i]);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        f[(int64_t)Q * ns + i] = S::template enc<Q>((typename S::M)d[(int64_t)Q * m.n + il], r_own);
    });
}
template <class S>
__global__ void k_batch_decode(const typename S::T* __restrict__ f, int64_t ns, const uint32_t* __restrict__ vox,
                               const Member* members, int mi, double* __restrict__ d) {
    const Member& m = members[mi];
    const int64_t il = (int64_t)blockIdx.x * kTile + threadIdx.x;
    if (il >= m.n) return;
    const int64_t i = m.base + il;
    const typename S::M r_own = member_ref<S>(m, vox[i]);
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[(int64_t)Q * m.n + il] = (double)S::template dec<Q>(f[(int64_t)Q * ns + i], r_own);
    });
}

// rho and u = j of one member's stored state into dense [z][y][x] arrays
// (pre-zeroed), via the member's unpadded voxel index list.
template <class S>
__global__ void k_batch_export(const typename S::T* __restrict__ f, int64_t ns, const uint32_t* __restrict__ vox,
                               const Member* members, int mi, const int64_t* __restrict__ unpadded, double* rho,
                               double* ux, double* uy, double* uz) {
    using M = typename S::M;
    const Member& m = members[mi];
    const int64_t il = (int64_t)blockIdx.x * kTile + threadIdx.x;
    if (il >= m.n) return;
    const int64_t i = m.base + il;
    const M r_own = member_ref<S>(m, vox[i]);
    M d[19];
    for_q(AllQ{}, [&](auto qc) {
        constexpr int Q = decltype(qc)::value;
        d[Q] = S::template dec<Q>(f[(int64_t)Q * ns + i], r_own);
    });
    M drho, jx, jy, jz;
    moments(d, drho, jx, jy, jz);
    const int64_t o = unpadded[il];
    rho[o] = 1.0 + (double)drho;
    ux[o] = (double)jx;
    uy[o] = (double)jy;
    uz[o] = (double)jz;
}

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

thread_local std::string g_batch_create_error;

}  // namespace
}  // namespace lbm

struct lbm_batch {
    int device = 0;
    int prec = 1;
    int nm = 0;
    double sp = 1.0, sm = 1.0;
    int64_t total = 0;   // global pore slots (multiple of the tile)
    int64_t ns = 0;      // row stride
    int64_t ntiles = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t* d_vox = nullptr;
    int* d_grid = nullptr;
    int* d_tile_member = nullptr;
    lbm::Member* d_members = nullptr;
    double* d_partials = nullptr;
    unsigned* d_counters = nullptr;    // one per member (step and inlet reductions)
    unsigned* d_counter1 = nullptr;    // face-flux reduction
    double* d_out = nullptr;
    std::vector<lbm::Member> h_members;
    std::vector<std::vector<int64_t>> pore_voxel;  // per member: unpadded voxel of each pore
    std::vector<int> dims;                          // 3 per member
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t steps = 0, since_reencode = 0;
    int ref_e = 0;
    int config = LBM_BATCH_GRAPH;      // launch form and register cap (lbm_batch_set_config)
    lbm::GridBarrier* d_bar = nullptr;  // grid barrier of the persistent launch
    int status = LBM_OK;
    std::string err;
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) {
        b->err = buf;
        if (code == LBM_ECUDA) b->status = LBM_ECUDA;
    } else {
        lbm::g_batch_create_error = buf;
    }
    return code;
}

#define BATCH_CUDA(b, call)                                                                \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail((b), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

int benter(lbm_batch* b) {
    if (!b) return LBM_EINVAL;
    if (b->status == LBM_ECUDA) return LBM_ECUDA;
    BATCH_CUDA(b, cudaSetDevice(b->device));
    return LBM_OK;
}

void brelease(lbm_batch* b) {
    for (auto& g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto& p : b->f)
        if (p) cudaFree(p);
    cudaFree(b->d_vox);
    cudaFree(b->d_grid);
    cudaFree(b->d_tile_member);
    cudaFree(b->d_members);
    cudaFree(b->d_partials);
    cudaFree(b->d_counters);
    cudaFree(b->d_counter1);
    cudaFree(b->d_out);
    cudaFree(b->d_bar);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}

// Register cap of a configuration: 4 or 5 resident 256-thread blocks per SM
// (64 or 48 registers).
constexpr bool cfg_capped(int cfg) {
    return cfg == LBM_BATCH_GRAPH_CAPPED || cfg == LBM_BATCH_PERSISTENT_CAPPED || cfg == LBM_BATCH_AA_CAPPED;
}
constexpr bool cfg_persistent(int cfg) { return cfg == LBM_BATCH_PERSISTENT || cfg == LBM_BATCH_PERSISTENT_CAPPED; }
constexpr bool cfg_aa(int cfg) { return cfg == LBM_BATCH_AA || cfg == LBM_BATCH_AA_CAPPED; }
// Buffer that holds the state: f[cur] for the pull forms, f[0] for the AA
// pattern (cur is then only the parity of the inlet-density slot).
void* bstate(lbm_batch* b) { return cfg_aa(b->config) ? b->f[0] : b->f[b->cur]; }
// Bounded wait of the persistent barrier: 2^31 SM cycles (about 1 s at 2 GHz).
constexpr long long kBarrierLimit = 1LL << 31;

template <class S, int MINB>
cudaError_t persistent_grid(int* grid, int64_t ntiles) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm::k_batch_persistent<S, MINB>,
                                                                  lbm::kTile, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *grid = (int)std::min<int64_t>((int64_t)per_sm * sms, ntiles);
    return cudaSuccess;
}

// `nsteps` steps in one cooperative launch (the persistent configurations).
int bpersistent(lbm_batch* b, int nsteps) {
    BATCH_CUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(lbm::GridBarrier), b->stream));
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        using T = typename S::T;
        using M = typename S::M;
        auto launch = [&](auto minb) -> cudaError_t {
            constexpr int MINB = decltype(minb)::value;
            int grid = 0;
            cudaError_t e2 = persistent_grid<S, MINB>(&grid, b->ntiles);
            if (e2 != cudaSuccess) return e2;
            T* f0 = (T*)b->f[0];
            T* f1 = (T*)b->f[1];
            int64_t ns = b->ns, ntiles = b->ntiles;
            int slot0 = b->cur, n = nsteps;
            M sp = (M)b->sp, sm = (M)b->sm;
            long long limit = kBarrierLimit;
            void* args[] = {&f0, &f1, &ns, &slot0, &n, &ntiles, &b->d_vox, &b->d_grid, &b->d_tile_member,
                            &b->d_members, &sp, &sm, &b->d_partials, &b->d_counters, &b->d_bar, &limit};
            return cudaLaunchCooperativeKernel((const void*)lbm::k_batch_persistent<S, MINB>, dim3(grid),
                                               dim3(lbm::kTile), args, 0, b->stream);
        };
        if (cfg_capped(b->config)) return launch(std::integral_constant<int, 5>{});
        return launch(std::integral_constant<int, 4>{});
    });
    BATCH_CUDA(b, e);
    if (nsteps & 1) b->cur ^= 1;
    return LBM_OK;
}

// The persistent launch records a barrier timeout in device memory.
int bcheck_barrier(lbm_batch* b) {
    lbm::GridBarrier h{};
    BATCH_CUDA(b, cudaMemcpyAsync(&h, b->d_bar, sizeof h, cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    if (h.err) return bfail(b, LBM_ETIMEOUT, "persistent launch: a block waited more than 2^31 cycles at the "
                                             "step barrier; the state of this call is incomplete");
    return LBM_OK;
}

int bstep_once(lbm_batch* b, cudaStream_t st) {
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        using T = typename S::T;
        using M = typename S::M;
        auto launch = [&](auto kernel) {
            kernel<<<(unsigned)b->ntiles, lbm::kTile, 0, st>>>(
                (const T*)b->f[b->cur], (T*)b->f[b->cur ^ 1], b->ns, b->cur, b->d_vox, b->d_grid,
                b->d_tile_member, b->d_members, (M)b->sp, (M)b->sm, b->d_partials, b->d_counters);
        };
        // every element offset of a buffer fits in 32 bits; GB300_LBM_BATCH_ADDR64 forces the 64-bit form (tests)
        const bool off32 = 19 * (uint64_t)b->ns <= 0xFFFFFFFFull && !std::getenv("GB300_LBM_BATCH_ADDR64");
        if (cfg_capped(b->config))
            off32 ? launch(lbm::k_batch_step<S, 5, true>) : launch(lbm::k_batch_step<S, 5>);
        else
            off32 ? launch(lbm::k_batch_step<S, 4, true>) : launch(lbm::k_batch_step<S, 4>);
        return cudaGetLastError();
    });
    BATCH_CUDA(b, e);
    b->cur ^= 1;
    return LBM_OK;
}

// One AA step of a call: gather-scatter when odd is set, node-local otherwise.
int bstep_aa(lbm_batch* b, cudaStream_t st, bool odd) {
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        using T = typename S::T;
        using M = typename S::M;
        auto go = [&](auto oddc, auto minbc) {
            constexpr bool ODD = decltype(oddc)::value;
            constexpr int MINB = decltype(minbc)::value;
            lbm::Rows<T> F;
            for (int q = 0; q < 19; ++q) F.row[q] = (T*)b->f[0] + (int64_t)q * b->ns;
            // OFF32 when every element offset fits in 32 bits
            if (19 * (uint64_t)b->ns <= 0xFFFFFFFFull && !std::getenv("GB300_LBM_BATCH_ADDR64"))
                lbm::k_batch_aa<S, ODD, MINB, true><<<(unsigned)b->ntiles, lbm::kTile, 0, st>>>(
                    F, b->cur, b->d_vox, b->d_grid, b->d_tile_member, b->d_members, (M)b->sp, (M)b->sm,
                    b->d_partials, b->d_counters);
            else
                lbm::k_batch_aa<S, ODD, MINB><<<(unsigned)b->ntiles, lbm::kTile, 0, st>>>(
                    F, b->cur, b->d_vox, b->d_grid, b->d_tile_member, b->d_members, (M)b->sp, (M)b->sm,
                    b->d_partials, b->d_counters);
        };
        const bool capped = cfg_capped(b->config);
        if (odd && capped) go(std::true_type{}, std::integral_constant<int, 5>{});
        else if (odd) go(std::true_type{}, std::integral_constant<int, 4>{});
        else if (capped) go(std::false_type{}, std::integral_constant<int, 5>{});
        else go(std::false_type{}, std::integral_constant<int, 4>{});
        return cudaGetLastError();
    });
    BATCH_CUDA(b, e);
    b->cur ^= 1;
    return LBM_OK;
}

int baa_layout(lbm_batch* b, bool unstream) {
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        using T = typename S::T;
        if (unstream)
            lbm::k_batch_aa_unstream<S><<<(unsigned)b->ntiles, lbm::kTile, 0, b->stream>>>(
                (T*)b->f[0], b->ns, b->d_vox, b->d_grid, b->d_tile_member, b->d_members);
        else
            lbm::k_batch_aa_swap<T><<<(unsigned)((b->total + 255) / 256), 256, 0, b->stream>>>((T*)b->f[0], b->total,
                                                                                             b->ns);
        return cudaGetLastError();
    });
    BATCH_CUDA(b, e);
    return LBM_OK;
}

int bprime(lbm_batch* b) {
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        using T = typename S::T;
        lbm::k_batch_inlet<S><<<(unsigned)b->ntiles, lbm::kTile, 0, b->stream>>>(
            (const T*)bstate(b), b->ns, b->cur, b->d_vox, b->d_grid, b->d_tile_member, b->d_members,
            b->d_partials, b->d_counters);
        return cudaGetLastError();
    });
    BATCH_CUDA(b, e);
    return LBM_OK;
}

int bmaybe_reencode(lbm_batch* b) {
    if (b->prec < LBM_PREC_FP16DEV || b->since_reencode < lbm::kBatchReencodeInterval) return LBM_OK;
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        using T = typename S::T;
        if constexpr (S::kRef) {
            lbm::k_batch_reencode<S><<<(unsigned)b->ntiles, lbm::kTile, 0, b->stream>>>(
                (T*)bstate(b), b->ns, b->d_vox, b->d_tile_member, b->d_members, b->ref_e, b->cur, b->total);
        }
        return cudaGetLastError();
    });
    BATCH_CUDA(b, e);
    b->ref_e ^= 1;
    b->since_reencode = 0;
    return bprime(b);
}

int bbuild_graph(lbm_batch* b, int parity) {
    const int saved = b->cur;
    b->cur = parity;
    cudaGraph_t g = nullptr;
    BATCH_CUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    for (int k = 0; k < lbm::kBatchGraphSteps && rc == LBM_OK; ++k)
        rc = cfg_aa(b->config) ? bstep_aa(b, b->cap_stream, (k & 1) == 0) : bstep_once(b, b->cap_stream);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    b->cur = saved;
    if (rc != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int push_member(lbm_batch* b, int mi) {
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_members + mi, &b->h_members[(size_t)mi], sizeof(lbm::Member),
                                  cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// Refresh the host copy of a member's device-side state (densities, profile).
int pull_member(lbm_batch* b, int mi) {
    BATCH_CUDA(b, cudaMemcpyAsync(&b->h_members[(size_t)mi], b->d_members + mi, sizeof(lbm::Member),
                                  cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int n_members, const uint8_t* const* masks, const int* dims, double tau, int model,
                     int precision, lbm_batch** out) {
    using lbm::g_batch_create_error;
    g_batch_create_error.clear();
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_members < 1 || n_members > 65535 || !masks || !dims)
        return bfail(nullptr, LBM_EINVAL, "need 1..65535 members with masks and dims");
    if (!(tau > 0.5) || !(tau < 1e6)) return bfail(nullptr, LBM_EINVAL, "tau=%g must exceed 0.5", tau);
    if (model != LBM_MODEL_BGK && model != LBM_MODEL_MRT) return bfail(nullptr, LBM_EINVAL, "unknown model");
    if (precision < LBM_PREC_FP64 || precision > LBM_PREC_BF16DEV)
        return bfail(nullptr, LBM_EINVAL, "unknown precision");
    auto* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation");
    cudaGetDevice(&b->device);
    b->prec = precision;
    b->nm = n_members;
    b->sp = 1.0 / tau;
    b->sm = model == LBM_MODEL_MRT ? 8.0 * (2.0 - b->sp) / (8.0 - b->sp) : b->sp;
    b->h_members.resize((size_t)n_members);
    b->pore_voxel.resize((size_t)n_members);
    b->dims.assign(dims, dims + 3 * n_members);

    std::vector<int> grid;
    std::vector<uint32_t> vox;
    std::vector<int> tile_member;
    int64_t base = 0, gbase = 0;
    for (int mi = 0; mi < n_members; ++mi) {
        const int nx = dims[3 * mi], ny = dims[3 * mi + 1], nz = dims[3 * mi + 2];
        const uint8_t* mask = masks[mi];
        if (!mask || nx < 1 || ny < 1 || nx > 2047 || ny > 2047 || nz < 3 || nz > 1023) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "member %d: bad mask or box %dx%dx%d", mi, nx, ny, nz);
        }
        const int64_t px = nx + 2, py = ny + 2, pz = nz + 2;
        const int64_t pad = px * py * pz;
        if (gbase + pad > (int64_t)UINT32_MAX) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "padded boxes exceed 2^32 voxels in total");
        }
        grid.resize((size_t)(gbase + pad), lbm::SOLID);
        for (int64_t y = 0; y < py; ++y)
            for (int64_t x = 0; x < px; ++x) {
                grid[(size_t)(gbase + y * px + x)] = lbm::ZOUT;
                grid[(size_t)(gbase + ((pz - 1) * py + y) * px + x)] = lbm::ZOUT;
            }
        lbm::Member m{};
        m.base = base;
        m.grid_base = gbase;
        m.nz = nz;
        int64_t a_in = 0, a_out = 0, a_01 = 0, n = 0;
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t v = (z * ny + y) * nx + x;
                    if (mask[v] > 1) {
                        delete b;
                        return bfail(nullptr, LBM_EINVAL, "member %d: mask value %d (must be 0 or 1)", mi, mask[v]);
                    }
                    if (mask[v]) continue;
                    const int64_t p = ((z + 1) * py + (y + 1)) * px + (x + 1);
                    grid[(size_t)(gbase + p)] = (int)(base + n);
                    vox.push_back((uint32_t)(gbase + p));
                    b->pore_voxel[(size_t)mi].push_back(v);
                    ++n;
                    if (z == 0) ++a_in;
                    if (z == nz - 1) ++a_out;
                    if (z <= 1) ++a_01;
                }
        if (a_in == 0 || a_out == 0) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "member %d: inlet and outlet planes need pore nodes", mi);
        }
        m.n = n;
        m.a_in = a_in;
        m.a_out = a_out;
        m.a_01 = a_01;
        for (int q = 0; q < 19; ++q) m.goff[q] = (int)(-(lbm::cz(q) * px * py + lbm::cy(q) * px + lbm::cx(q)));
        const unsigned __int128 two64 = (unsigned __int128)1 << 64;
        const unsigned __int128 szq = (unsigned __int128)(uint64_t)(px * py);
        m.sz_magic = (uint64_t)(two64 / szq + (two64 % szq != 0 ? 1 : 0));
        b->h_members[(size_t)mi] = m;
        const int64_t nt = (n + lbm::kTile - 1) / lbm::kTile;
        for (int64_t t = 0; t < nt; ++t) tile_member.push_back(mi);
        vox.resize((size_t)(base + nt * lbm::kTile), 0u);
        base += nt * lbm::kTile;
        gbase += pad;
        if (base >= INT32_MAX) {
            delete b;
            return bfail(nullptr, LBM_EINVAL, "more than 2^31-1 pore slots in total");
        }
    }
    b->total = base;
    b->ntiles = base / lbm::kTile;
    b->ns = (base + 127) / 128 * 128;
    const size_t fbytes = (size_t)19 * (size_t)b->ns * (size_t)lbm::elem_size(precision);
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
    };
    A(&b->f[0], fbytes);
    A(&b->f[1], fbytes);
    A(&b->d_vox, vox.size() * 4);
    A(&b->d_grid, grid.size() * 4);
    A(&b->d_tile_member, tile_member.size() * 4);
    A(&b->d_members, (size_t)n_members * sizeof(lbm::Member));
    A(&b->d_partials, (size_t)b->ntiles * sizeof(double));
    A(&b->d_counters, (size_t)n_members * sizeof(unsigned));
    A(&b->d_counter1, sizeof(unsigned));
    A(&b->d_out, sizeof(double));
    A(&b->d_bar, sizeof(lbm::GridBarrier));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_vox, vox.data(), vox.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_grid, grid.data(), grid.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_tile_member, tile_member.data(), tile_member.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_members, b->h_members.data(), (size_t)n_members * sizeof(lbm::Member),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, (size_t)n_members * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_counter1, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, sizeof(lbm::GridBarrier));
    // rest state: d = f - w = 0 in every format (the reference profile starts at 0)
    if (e == cudaSuccess) e = cudaMemset(b->f[0], 0, fbytes);
    if (e == cudaSuccess) e = cudaMemset(b->f[1], 0, fbytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "lbm_batch_create: %s",
              cudaGetErrorString(e));
        cudaGetLastError();
        brelease(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
    int rc = bprime(b);
    if (rc == LBM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = LBM_ECUDA;
    if (rc != LBM_OK) {
        g_batch_create_error = b->err;
        brelease(b);
        delete b;
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch* b, void* s) {
    int rc = benter(b);
    if (rc) return rc;
    b->stream = (cudaStream_t)s;
    return LBM_OK;
}

int lbm_batch_set_flux_bc(lbm_batch* b, int member, double Q) {
    int rc = benter(b);
    if (rc) return rc;
    if (member < 0 || member >= b->nm) return bfail(b, LBM_EINVAL, "member %d out of range", member);
    if (!(Q == Q) || Q > 1e30 || Q < -1e30) return bfail(b, LBM_EINVAL, "Q must be finite");
    if ((rc = pull_member(b, member))) return rc;
    b->h_members[(size_t)member].Q = Q;
    if ((rc = push_member(b, member))) return rc;
    return bprime(b);
}

int lbm_batch_step(lbm_batch* b, int n) {
    int rc = benter(b);
    if (rc) return rc;
    if (n < 0) return bfail(b, LBM_EINVAL, "n must be >= 0");
    if (cfg_aa(b->config)) {
        // segments end at the 16-bit reference refreshes, which work on the pull layout
        int64_t k = 0;
        while (k < n) {
            if ((rc = bmaybe_reencode(b))) return rc;
            int64_t seg = n - k;
            if (b->prec >= LBM_PREC_FP16DEV) seg = std::min<int64_t>(seg, lbm::kBatchReencodeInterval - b->since_reencode);
            if ((rc = baa_layout(b, false))) return rc;
            int64_t j = 0;
            while (seg - j >= lbm::kBatchGraphSteps) {
                if (!b->graph[b->cur] && (rc = bbuild_graph(b, b->cur))) return rc;
                BATCH_CUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
                j += lbm::kBatchGraphSteps;
            }
            for (; j < seg; ++j)
                if ((rc = bstep_aa(b, b->stream, (j & 1) == 0))) return rc;
            if ((seg & 1) && (rc = baa_layout(b, true))) return rc;
            if ((rc = baa_layout(b, false))) return rc;
            k += seg;
            b->since_reencode += seg;
        }
        b->steps += n;
        return LBM_OK;
    }
    if (cfg_persistent(b->config)) {
        // one cooperative launch per segment between 16-bit reference refreshes
        int64_t k = 0;
        while (k < n) {
            if ((rc = bmaybe_reencode(b))) return rc;
            int64_t seg = n - k;
            if (b->prec >= LBM_PREC_FP16DEV) seg = std::min<int64_t>(seg, lbm::kBatchReencodeInterval - b->since_reencode);
            if ((rc = bpersistent(b, (int)seg))) return rc;
            k += seg;
            b->since_reencode += seg;
        }
        if (n > 0 && (rc = bcheck_barrier(b))) return rc;
        b->steps += n;
        return LBM_OK;
    }
    int k = 0;
    while (n - k >= lbm::kBatchGraphSteps) {
        if ((rc = bmaybe_reencode(b))) return rc;
        if (!b->graph[b->cur] && (rc = bbuild_graph(b, b->cur))) return rc;
        BATCH_CUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
        k += lbm::kBatchGraphSteps;
        b->since_reencode += lbm::kBatchGraphSteps;
    }
    for (; k < n; ++k) {
        if ((rc = bmaybe_reencode(b))) return rc;
        if ((rc = bstep_once(b, b->stream))) return rc;
        ++b->since_reencode;
    }
    b->steps += n;
    return LBM_OK;
}

int lbm_batch_time_step(lbm_batch* b, int n, float* ms) {
    int rc = benter(b);
    if (rc) return rc;
    if (n < 1) return bfail(b, LBM_EINVAL, "n must be >= 1");
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    BATCH_CUDA(b, cudaEventCreate(&e1));
    double tot = 0.0;
    if (cfg_persistent(b->config)) {
        BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
        if ((rc = bpersistent(b, n))) return rc;
        BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
        BATCH_CUDA(b, cudaEventSynchronize(e1));
        float t = 0.f;
        BATCH_CUDA(b, cudaEventElapsedTime(&t, e0, e1));
        tot = t;
        if ((rc = bcheck_barrier(b))) return rc;
    }
    if (cfg_aa(b->config)) {
        // the AA steps of one call (the layout swaps included)
        BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
        if ((rc = lbm_batch_step(b, n))) return rc;
        BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
        BATCH_CUDA(b, cudaEventSynchronize(e1));
        float t = 0.f;
        BATCH_CUDA(b, cudaEventElapsedTime(&t, e0, e1));
        tot = t;
        b->steps -= n;  // counted below
        b->since_reencode -= n;
    }
    for (int k = 0; k < n && !cfg_persistent(b->config) && !cfg_aa(b->config); ++k) {
        BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
        if ((rc = bstep_once(b, b->stream))) return rc;
        BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
        BATCH_CUDA(b, cudaEventSynchronize(e1));
        float t = 0.f;
        BATCH_CUDA(b, cudaEventElapsedTime(&t, e0, e1));
        tot += t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->steps += n;
    b->since_reencode += n;
    if (ms) *ms = (float)(tot / n);
    return LBM_OK;
}

int lbm_batch_get_flux(lbm_batch* b, int member, int face, double* Q, double* rho_bc) {
    int rc = benter(b);
    if (rc) return rc;
    if (member < 0 || member >= b->nm) return bfail(b, LBM_EINVAL, "member %d out of range", member);
    if (face != LBM_FACE_ZMIN && face != LBM_FACE_ZMAX) return bfail(b, LBM_EINVAL, "unknown face %d", face);
    if ((rc = pull_member(b, member))) return rc;
    const lbm::Member& m = b->h_members[(size_t)member];
    const unsigned nt = (unsigned)((m.n + lbm::kTile - 1) / lbm::kTile);
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        lbm::k_batch_face_flux<S><<<nt, lbm::kTile, 0, b->stream>>>(
            (const typename S::T*)bstate(b), b->ns, b->d_vox, b->d_members, member,
            face == LBM_FACE_ZMIN ? 0 : 1, b->d_partials, b->d_counter1, b->d_out);
        return cudaGetLastError();
    });
    BATCH_CUDA(b, e);
    double q = 0.0;
    BATCH_CUDA(b, cudaMemcpyAsync(&q, b->d_out, sizeof q, cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    if (Q) *Q = q;
    if (rho_bc) *rho_bc = 1.0 + (face == LBM_FACE_ZMAX ? m.drho_out : m.drho_in[b->cur ^ 1]);
    return LBM_OK;
}

int lbm_batch_get_distributions(lbm_batch* b, int member, double* f) {
    int rc = benter(b);
    if (rc) return rc;
    if (member < 0 || member >= b->nm || !f) return bfail(b, LBM_EINVAL, "bad member or NULL f");
    const lbm::Member& m = b->h_members[(size_t)member];
    const size_t ncell = (size_t)b->dims[3 * member] * b->dims[3 * member + 1] * b->dims[3 * member + 2];
    std::vector<double> h((size_t)(19 * m.n));
    double* d = nullptr;
    BATCH_CUDA(b, cudaMalloc(&d, h.size() * sizeof(double)));
    cudaError_t e = lbm::dispatch(b->prec, [&](auto s) {
        using S = decltype(s);
        lbm::k_batch_decode<S><<<(unsigned)((m.n + lbm::kTile - 1) / lbm::kTile), lbm::kTile, 0, b->stream>>>(
            (const typename S::T*)bstate(b), b->ns, b->d_vox, b->d_members, member, d);
        return cudaGetLastError();
    });
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_get_distributions: %s", cudaGetErrorString(e));
    std::memset(f, 0, 19 * ncell * sizeof(double));
    const auto& pv = b->pore_voxel[(size_t)member];
    for (int q = 0; q < 19; ++q)
        for (int64_t i = 0; i < m.n; ++i)
            f[(size_t)q * ncell + (size_t)pv[(size_t)i]] = lbm::wq(q) + h[(size_t)(q * m.n + i)];
    return LBM_OK;
}

int lbm_batch_set_distributions(lbm_batch* b, int member, const double* f) {
    int rc = benter(b);
    if (rc) return rc;
    if (member < 0 || member >= b->nm || !f) return bfail(b, LBM_EINVAL, "bad member or NULL f");
    if ((rc = pull_member(b, member))) return rc;
    const lbm::Member& m = b->h_members[(size_t)member];
    const size_t ncell = (size_t)b->dims[3 * member] * b->dims[3 * member + 1] * b->dims[3 * member + 2];
    const auto& pv = b->pore_voxel[(size_t)member];
    std::vector<double> h((size_t)(19 * m.n));
    for (int q = 0; q < 19; ++q)
        for (int64_t i = 0; i < m.n; ++i)
            h[(size_t)(q * m.n + i)] = f[(size_t)q * ncell + (size_t)pv[(size_t)i]] - lbm::wq(q);
    double* d = nullptr;
    BATCH_CUDA(b, cudaMalloc(&d, h.size() * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = lbm::dispatch(b->prec, [&](auto s) {
            using S = decltype(s);
            lbm::k_batch_encode<S><<<(unsigned)((m.n + lbm::kTile - 1) / lbm::kTile), lbm::kTile, 0, b->stream>>>(
                (typename S::T*)bstate(b), b->ns, b->d_vox, b->d_members, member, d);
            return cudaGetLastError();
        });
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_set_distributions: %s", cudaGetErrorString(e));
    return bprime(b);
}

int lbm_batch_get_fields(lbm_batch* b, int member, double* rho, double* ux, double* uy, double* uz) {
    int rc = benter(b);
    if (rc) return rc;
    if (member < 0 || member >= b->nm) return bfail(b, LBM_EINVAL, "member %d out of range", member);
    const lbm::Member& m = b->h_members[(size_t)member];
    const size_t ncell = (size_t)b->dims[3 * member] * b->dims[3 * member + 1] * b->dims[3 * member + 2];
    const auto& pv = b->pore_voxel[(size_t)member];
    double* d = nullptr;
    int64_t* dv = nullptr;
    BATCH_CUDA(b, cudaMalloc(&d, 4 * ncell * sizeof(double)));
    cudaError_t e = cudaMalloc(&dv, pv.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, 4 * ncell * sizeof(double), b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dv, pv.data(), pv.size() * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = lbm::dispatch(b->prec, [&](auto s) {
            using S = decltype(s);
            lbm::k_batch_export<S><<<(unsigned)((m.n + lbm::kTile - 1) / lbm::kTile), lbm::kTile, 0, b->stream>>>(
                (const typename S::T*)bstate(b), b->ns, b->d_vox, b->d_members, member, dv, d, d + ncell,
                d + 2 * ncell, d + 3 * ncell);
            return cudaGetLastError();
        });
    double* outs[4] = {rho, ux, uy, uz};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (outs[k])
            e = cudaMemcpyAsync(outs[k], d + k * ncell, ncell * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    cudaFree(dv);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_get_fields: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_batch_get_info(const lbm_batch* b, int64_t* n_pore, int64_t* n_tiles, int64_t* steps) {
    if (!b) return LBM_EINVAL;
    int64_t n = 0;
    for (const auto& m : b->h_members) n += m.n;
    if (n_pore) *n_pore = n;
    if (n_tiles) *n_tiles = b->ntiles;
    if (steps) *steps = b->steps;
    return LBM_OK;
}

int lbm_batch_set_config(lbm_batch* b, int config) {
    int rc = benter(b);
    if (rc) return rc;
    if (config < 0 || config >= LBM_BATCH_NCONFIG) return bfail(b, LBM_EINVAL, "unknown configuration %d", config);
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    // the AA pattern keeps the state in f[0]: move it between f[0] and f[cur]
    if (cfg_aa(b->config) != cfg_aa(config) && b->cur == 1) std::swap(b->f[0], b->f[1]);
    b->config = config;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* best, float* ms_per_step) {
    int rc = benter(b);
    if (rc) return rc;
    if (trial_steps < 1) return bfail(b, LBM_EINVAL, "trial_steps must be >= 1");
    const size_t fbytes = (size_t)19 * (size_t)b->ns * (size_t)(b->prec == 0 ? 8 : b->prec == 1 ? 4 : 2);
    void* backup = nullptr;
    if (cudaMalloc(&backup, fbytes) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LBM_ENOMEM, "lbm_batch_autotune: no room for a copy of the state (%zu bytes)", fbytes);
    }
    // the trials start from, and leave behind, the state of this call
    const int cur0 = b->cur, ref_e0 = b->ref_e, cfg0 = b->config;
    const int64_t steps0 = b->steps, since0 = b->since_reencode;
    auto save_restore = [&](bool save) -> int {
        if (save) {
            BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
            BATCH_CUDA(b, cudaMemcpy(backup, bstate(b), fbytes, cudaMemcpyDeviceToDevice));
            BATCH_CUDA(b, cudaMemcpy(b->h_members.data(), b->d_members, (size_t)b->nm * sizeof(lbm::Member),
                                     cudaMemcpyDeviceToHost));
        } else {
            BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
            b->cur = cur0;
            BATCH_CUDA(b, cudaMemcpy(bstate(b), backup, fbytes, cudaMemcpyDeviceToDevice));
            BATCH_CUDA(b, cudaMemcpy(b->d_members, b->h_members.data(), (size_t)b->nm * sizeof(lbm::Member),
                                     cudaMemcpyHostToDevice));
            b->ref_e = ref_e0;
            b->steps = steps0;
            b->since_reencode = since0;
        }
        return LBM_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float t[LBM_BATCH_NCONFIG];
    int choice = cfg0;
    rc = save_restore(true);
    if (rc == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = bfail(b, LBM_ECUDA, "lbm_batch_autotune: event creation failed");
    for (int c = 0; c < LBM_BATCH_NCONFIG && rc == LBM_OK; ++c) {
        if ((rc = lbm_batch_set_config(b, c))) break;
        // untimed run first: graph capture and first-launch costs
        if ((rc = lbm_batch_step(b, trial_steps)) || (rc = save_restore(false))) break;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) { rc = bfail(b, LBM_ECUDA, "event record"); break; }
        if ((rc = lbm_batch_step(b, trial_steps))) break;
        if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t[c], e0, e1) != cudaSuccess) {
            rc = bfail(b, LBM_ECUDA, "event timing");
            break;
        }
        t[c] /= (float)trial_steps;
        if ((rc = save_restore(false))) break;
        if (t[c] < t[choice] || c == 0) choice = c;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(backup);
    if (rc != LBM_OK) return rc;
    if ((rc = lbm_batch_set_config(b, choice))) return rc;
    if (best) *best = choice;
    if (ms_per_step)
        for (int c = 0; c < LBM_BATCH_NCONFIG; ++c) ms_per_step[c] = t[c];
    return LBM_OK;
}

int lbm_batch_check_barrier(lbm_batch* b, double timeout_ms, int* completes, int* times_out) {
    int rc = benter(b);
    if (rc) return rc;
    if (!(timeout_ms > 0.0) || timeout_ms > 2000.0) return bfail(b, LBM_EINVAL, "timeout_ms must be in (0, 2000]");
    const long long limit = (long long)(timeout_ms * 2.1e6);  // cycles at up to 2.1 GHz
    int got[2] = {0, 0};
    for (int k = 0; k < 2; ++k) {
        lbm::GridBarrier h{};
        BATCH_CUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof h, b->stream));
        lbm::k_barrier_probe<<<4, 32, 0, b->stream>>>(b->d_bar, k == 0 ? 4u : 5u, limit);
        BATCH_CUDA(b, cudaGetLastError());
        BATCH_CUDA(b, cudaMemcpyAsync(&h, b->d_bar, sizeof h, cudaMemcpyDeviceToHost, b->stream));
        BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
        got[k] = h.err;
    }
    BATCH_CUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(lbm::GridBarrier), b->stream));
    if (completes) *completes = got[0] == 0;
    if (times_out) *times_out = got[1] != 0;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    brelease(b);
    delete b;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) {
    return b ? b->err.c_str() : lbm::g_batch_create_error.c_str();
}

}  // extern "C"
