// Device-side building blocks of the D3Q19 flux-boundary solver: the lattice,
// the storage codecs, the pull gather, the boundary closures and the collision.
//
// State convention: the device holds the shifted distributions
//     d_q = f_q - w_q
// (the deviation from the rest-state weight).  Every formula of the method is
// affine in f with weight sums that cancel, so it is evaluated on d with the
// density replaced by drho = rho - 1 (see each function).  This keeps the
// significant digits of the small deviations in every storage format.
#pragma once

#include <cstddef>
#include <cstdint>
#include <utility>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbm {

// ---------------------------------------------------------------- lattice ---
// Eq. (d3q19): q = 0 rest; 1..6 = +-x, +-y, +-z; 7..18 diagonals in the order
// for which the Appendix B momentum rows hold: 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0)
// 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1)
// 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1).  Opposites pair as (odd q, q+1).
__host__ __device__ constexpr int cx(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
         : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
         : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
         : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
// weights: 1/3 rest, 1/18 axes, 1/36 diagonals (c_s^2 = 1/3)
__host__ __device__ constexpr double wq(int q) {
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Padded voxel-id grid entries (see the host side): >= 0 pore index,
// SOLID for a solid or lateral out-of-box voxel, ZOUT outside the box in z.
constexpr int SOLID = -1;
constexpr int ZOUT = -2;

// ----------------------------------------------------------------- codecs ---
// Storage of d_q.  FP64 / FP32 store d_q.  The 16-bit formats store
//     (d_q / w_q - r) * 2^10 = (f_q / w_q - 1 - r) * 2^10,
// the deviation from the weight scaled to the reference density 1 + r of the
// plane z of the node that WROTE the value, r = r0 + g z (a linear profile
// between the inlet and outlet densities, refreshed by re-encoding).  Removing
// the mean pressure gradient leaves the local deviation, so the 11 (FP16) or 8
// (BF16) significant bits resolve the velocity part instead of the density ramp.
//
// The steps store the 16-bit formats with stochastic rounding (enc_sr): a value
// is rounded up in magnitude with probability equal to its distance from the
// lower neighbour in units of the last place, so the rounding error has zero
// mean.  Round-to-nearest would repeat the same error every step once the flow
// is steady and bias the steady state.  The random bits come from a
// counter-based hash of (step seed, node), so a run is reproducible.  Format
// conversions (encode, refresh) round to nearest.
//
// The rounding is the conversion instruction cvt.rs.{f16x2,bf16x2}.f32 (PTX ISA
// 8.7, sm_100a and later): it converts two FP32 values into one packed pair,
// adding the bits of its 32-bit rbits operand to the discarded low bits of each
// magnitude and truncating.  Lane layout (measured on sm_103a with values
// placed exactly below a rounding boundary, one rbits bit set at a time): the
// value in the upper half takes rbits bits 16-28 (FP16: 13 discarded bits) or
// 16-31 (BF16: 16), the value in the lower half bits 0-12 or 0-15; each half
// depends on its own input only.  enc_sr2 rounds both values of an opposite
// pair (q odd, q + 1) with one instruction.
//
// LBM_SR_MODE chooses the random numbers of a node's 19 values:
//   2 (default): one random number per node for all 19 values;
//   1: one per opposite pair, its two values on disjoint bit fields;
//   0: one per direction (h + q * phi) * C, its top bits, as the conversion-
//      free encode (add the bits, truncate) used before; gives identical states.
// Each value is rounded without bias in every mode; what differs is how the
// errors of a node's values are correlated.  With one number per node, an
// opposite pair's errors are positively correlated (a large number rounds both
// up), so they partly cancel in the momentum sum_q xi_q d_q.  Measured on a
// 128^3 pack, 5000 steps from the FP64 steady state, L2 / max velocity error
// against FP64: FP16-dev 3.7e-4 / 1.6e-3 (mode 2), 5.7e-4 / 7.2e-3 (mode 1),
// 3.8e-4 / 2.9e-3 (mode 0); BF16-dev 3.0e-3 / 2.7e-2, 4.7e-3 / 5.9e-2,
// 3.1e-3 / 2.6e-2; permeability within 6e-5 in all.  Mode 2 also needs no
// per-value key arithmetic (FP16-dev AA step 0.1617 ms against 0.1660 and 0.1761).
#ifndef LBM_SR_MODE
#define LBM_SR_MODE 2
#endif
constexpr bool kSrSameField = LBM_SR_MODE == 2;
constexpr float DEV_SCALE = 1024.0f;
// Half of the packed stochastic conversion that direction q uses.
__host__ __device__ constexpr bool sr_upper(int q) { return q == 0 || (q & 1); }

// 32-bit integer hash: the "lowbias32" finaliser published by C. Wellons
// (xor-shift / multiply rounds).
__host__ __device__ __forceinline__ uint32_t sr_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
// Seed of the next step.
__host__ __device__ __forceinline__ uint32_t sr_next(uint32_t seed) { return sr_hash(seed + 0x9E3779B9U); }

struct StoreF64 {
    using T = double;
    using M = double;
    static constexpr bool kRef = false;
    template <int Q> __device__ static M dec(T v, M) { return v; }
    template <int Q> __device__ static T enc(M v, M) { return v; }
    template <int Q> __device__ static T enc_sr(M v, M, uint32_t) { return v; }
};
struct StoreF32 {
    using T = float;
    using M = float;
    static constexpr bool kRef = false;
    template <int Q> __device__ static M dec(T v, M) { return v; }
    template <int Q> __device__ static T enc(M v, M) { return v; }
    template <int Q> __device__ static T enc_sr(M v, M, uint32_t) { return v; }
};
struct StoreF16 {
    using T = __half;
    using M = float;
    static constexpr bool kRef = true;
    // one fused multiply-add each way; w r and 1024 r take few distinct values per
    // node (3 weights, 3 planes), so the compiler forms them once
    template <int Q> __device__ static M dec(T v, M r) {
        return fmaf(__half2float(v), float(wq(Q) / 1024.0), float(wq(Q)) * r);
    }
    template <int Q> __device__ static T enc(M v, M r) {
        return __float2half_rn(fmaf(v, float(1024.0 / wq(Q)), -1024.0f * r));
    }
    // stochastic rounding of the values of Q (upper half) and Q + 1 (lower half)
    __device__ static uint32_t cvt_rs(float hi, float lo, uint32_t u) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(u));
        return d;
    }
    __device__ static T half_of(uint32_t d, bool upper) {
        return __ushort_as_half((unsigned short)(upper ? d >> 16 : d & 0xFFFFu));
    }
    template <int Q> __device__ static float scaled(M v, M r) { return fmaf(v, float(1024.0 / wq(Q)), -1024.0f * r); }
    // rbits of the upper / lower half from a key (13-bit fields at bits 16 and 0)
    __device__ static uint32_t bits_hi(uint32_t u) { return LBM_SR_MODE == 0 ? u >> 3 : u; }
    __device__ static uint32_t bits_lo(uint32_t u) { return LBM_SR_MODE == 0 ? u >> 19 : u; }
    template <int Q> __device__ static T enc_sr(M v, M r, uint32_t u) {
        constexpr bool up = sr_upper(Q) && !kSrSameField;
        return half_of(up ? cvt_rs(scaled<Q>(v, r), 0.0f, bits_hi(u)) : cvt_rs(0.0f, scaled<Q>(v, r), bits_lo(u)), up);
    }
    template <int Q> __device__ static uint32_t enc_sr2(M v, M r, M v1, M r1, uint32_t u, uint32_t u1) {
        static_assert(Q & 1, "a pair starts at an odd direction");
        return cvt_rs(scaled<Q>(v, r), scaled<Q + 1>(v1, r1),
                      LBM_SR_MODE == 0 ? ((bits_hi(u) & 0xFFFF0000u) | bits_lo(u1)) : u);
    }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    using M = float;
    static constexpr bool kRef = true;
    template <int Q> __device__ static M dec(T v, M r) {
        return fmaf(__bfloat162float(v), float(wq(Q) / 1024.0), float(wq(Q)) * r);
    }
    template <int Q> __device__ static T enc(M v, M r) {
        return __float2bfloat16_rn(fmaf(v, float(1024.0 / wq(Q)), -1024.0f * r));
    }
    __device__ static uint32_t cvt_rs(float hi, float lo, uint32_t u) {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(u));
        return d;
    }
    __device__ static T half_of(uint32_t d, bool upper) {
        return __ushort_as_bfloat16((unsigned short)(upper ? d >> 16 : d & 0xFFFFu));
    }
    template <int Q> __device__ static float scaled(M v, M r) { return fmaf(v, float(1024.0 / wq(Q)), -1024.0f * r); }
    // rbits of the upper / lower half from a key (16-bit fields at bits 16 and 0)
    __device__ static uint32_t bits_hi(uint32_t u) { return u; }
    __device__ static uint32_t bits_lo(uint32_t u) { return LBM_SR_MODE == 0 ? u >> 16 : u; }
    template <int Q> __device__ static T enc_sr(M v, M r, uint32_t u) {
        constexpr bool up = sr_upper(Q) && !kSrSameField;
        return half_of(up ? cvt_rs(scaled<Q>(v, r), 0.0f, bits_hi(u)) : cvt_rs(0.0f, scaled<Q>(v, r), bits_lo(u)), up);
    }
    template <int Q> __device__ static uint32_t enc_sr2(M v, M r, M v1, M r1, uint32_t u, uint32_t u1) {
        static_assert(Q & 1, "a pair starts at an odd direction");
        return cvt_rs(scaled<Q>(v, r), scaled<Q + 1>(v1, r1),
                      LBM_SR_MODE == 0 ? ((u & 0xFFFF0000u) | bits_lo(u1)) : u);
    }
};

// Random bits of the stochastic rounding of value (node i, direction q) in the
// step with seed `seed` (no work for the formats that store exactly): one hash
// per node (the same call for every q, computed once).  Mode 2 places its upper
// 16 bits in both halves of the rbits word, so either half of a conversion
// draws the same number; modes 0 and 1 add a Weyl step per direction or pair
// and mix it by one multiply.
template <class S>
__device__ __forceinline__ uint32_t sr_key(uint32_t seed, int64_t i, int q) {
    if constexpr (S::kRef) {
        const uint32_t h = sr_hash(seed ^ (uint32_t)i);
        if constexpr (LBM_SR_MODE == 2) {
            (void)q;
            return __byte_perm(h, 0u, 0x3232u);
        } else {
            return (h + (uint32_t)(LBM_SR_MODE == 1 ? (q + 1) >> 1 : q) * 0x9E3779B9U) * 0x2C1B3C6DU;
        }
    } else {
        return 0u;
    }
}

// Encodes the 19 values d of a node and hands each to put(Q, value), Q an
// std::integral_constant; ref(Q) is the reference density of the plane that
// direction Q's value is stored for (16-bit formats).  The 16-bit formats round
// the two values of each opposite pair (q odd, q + 1) with one conversion.
template <class S, int Q, class Ref, class Put>
__device__ __forceinline__ void encode_pair_(const typename S::M* d, uint32_t seed, int64_t i, Ref& ref, Put& put) {
    using C0 = std::integral_constant<int, Q>;
    using C1 = std::integral_constant<int, Q + 1>;
    const uint32_t u = sr_key<S>(seed, i, Q);
    if constexpr (S::kRef) {
        const uint32_t h = S::template enc_sr2<Q>(d[Q], ref(C0{}), d[Q + 1], ref(C1{}), u, sr_key<S>(seed, i, Q + 1));
        put(C0{}, S::half_of(h, true));
        put(C1{}, S::half_of(h, false));
    } else {
        put(C0{}, S::template enc_sr<Q>(d[Q], ref(C0{}), u));
        put(C1{}, S::template enc_sr<Q + 1>(d[Q + 1], ref(C1{}), u));
    }
}
template <class S, class Ref, class Put, int... P>
__device__ __forceinline__ void encode_node_(const typename S::M* d, uint32_t seed, int64_t i, Ref& ref, Put& put,
                                             std::integer_sequence<int, P...>) {
    using C0 = std::integral_constant<int, 0>;
    put(C0{}, S::template enc_sr<0>(d[0], ref(C0{}), sr_key<S>(seed, i, 0)));
    (encode_pair_<S, 2 * P + 1>(d, seed, i, ref, put), ...);
}
template <class S, class Ref, class Put>
__device__ __forceinline__ void encode_node(const typename S::M* d, uint32_t seed, int64_t i, Ref&& ref, Put&& put) {
    encode_node_<S>(d, seed, i, ref, put, std::make_integer_sequence<int, 9>{});
}

// ------------------------------------------------------- boundary state ---
// FP64 scalars of the boundary conditions, in device memory so that captured
// graphs pick up new values.  All densities are stored as drho = rho - 1.
// drho_in[c] is the inlet density (Eq. potential) for the step that reads
// distribution buffer c; the step that reads buffer c produces drho_in[c ^ 1].
struct BcState {
    double Q;              // prescribed inlet flux (Eq. flux)
    double drho_in_fixed;  // inlet density when the inlet is in pressure mode
    double drho_out;       // outlet density
    int inlet_mode;        // 0 = flux (Eq. potential), 1 = fixed pressure
    int pad_;
    double drho_in[2];     // per buffer parity, see above
    // Reference density profile r(z) = r0 + g z of the 16-bit formats, two
    // slots: ref_cur selects the one the stored values are encoded with.
    float ref_r0[2];
    float ref_g[2];
    int ref_cur;
    // stochastic-rounding seed of the step reading buffer c (16-bit formats)
    uint32_t sr_seed[2];
    int pad2_;
};
// The host writes only the fields before drho_in; the rest is device-owned.
constexpr size_t kBcHostBytes = offsetof(BcState, drho_in);

// Plane z of a padded voxel index p = ((z+1)(ny+2) + y+1)(nx+2) + x+1, with
// magic = ceil(2^64 / ((nx+2)(ny+2))): exact for p < 2^32.
__device__ __forceinline__ int plane_of(uint64_t p, uint64_t magic) {
    return (int)__umul64hi(p, magic) - 1;
}
template <class M>
__device__ __forceinline__ M ref_at(const BcState* bc, int z) {
    const int c = bc->ref_cur;
    return M(bc->ref_r0[c]) + M(bc->ref_g[c]) * M(z);
}
template <class M>
__device__ __forceinline__ M ref_slope(const BcState* bc) {
    return M(bc->ref_g[bc->ref_cur]);
}

// ------------------------------------------------------- cache hints ---
// L2 eviction-priority hints (PTX createpolicy / .L2::cache_hint): the streamed
// distributions are marked evict-first, the small index structures (id grid,
// voxel list) evict-last, so the latter stay in L2 from one step to the next.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Bulk L2 prefetch (cp.async.bulk.prefetch.L2, sm_90 and later) of the elements
// [s, min(s + len, end)) of an array that starts on a 16-byte boundary: the lines
// are fetched into L2 in the background and nothing waits for them.  The caller
// keeps s and end multiples of 16 / sizeof(T) elements, so that the byte offset
// and the size are multiples of 16 (a misaligned bulk copy is an illegal
// instruction).  Rows of ns elements, ns a multiple of 128, keep any row start
// aligned for every element size used here.
template <class T>
__device__ __forceinline__ void l2_prefetch_range(const T* base, int64_t s, int64_t len, int64_t end) {
    if (s < end) {
        const int64_t e = s + len < end ? s + len : end;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(base + s)),
                     "r"((uint32_t)((e - s) * (int64_t)sizeof(T))));
    }
}
__device__ __forceinline__ double ld_hint(const double* a, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_hint(const float* a, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ __half ld_hint(const __half* a, uint64_t pol) {
    unsigned short v;
    asm("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(pol));
    return __ushort_as_half(v);
}
__device__ __forceinline__ __nv_bfloat16 ld_hint(const __nv_bfloat16* a, uint64_t pol) {
    unsigned short v;
    asm("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(pol));
    return __ushort_as_bfloat16(v);
}
__device__ __forceinline__ int ld_hint(const int* a, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned ld_hint(const unsigned* a, uint64_t pol) {
    unsigned v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(double* a, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(float* a, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(__half* a, __half v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(a), "h"(__half_as_ushort(v)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_hint(__nv_bfloat16* a, __nv_bfloat16 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(a), "h"(__bfloat16_as_ushort(v)),
                 "l"(pol)
                 : "memory");
}

// ------------------------------------------------------------ helpers ---
template <int Q>
__device__ __forceinline__ int64_t grid_off(int sy, int sz) {
    // padded-grid offset of the pull source x - xi_q
    return -((int64_t)cz(Q) * sz + (int64_t)cy(Q) * sy + cx(Q));
}

// Pull one direction: d~_q(i) = d_q(src) for a pore source, own d_opp(i) for a
// solid (halfway bounce-back) or z-outside source (overwritten by the closure).
// r_own / g: reference profile at the node's plane and its slope; a pulled
// value was written on plane z - xi_z, where the reference is r_own - g xi_z.
template <class S, int Q>
__device__ __forceinline__ typename S::M pull(const typename S::T* __restrict__ fin, int64_t ns,
                                              const int* __restrict__ grid, int64_t p, int i,
                                              int sy, int sz, typename S::M r_own, typename S::M g) {
    using M = typename S::M;
    if (Q == 0) return S::template dec<0>(fin[i], r_own);
    const int id = __ldg(grid + p + grid_off<Q>(sy, sz));
    if (id >= 0) return S::template dec<Q>(fin[(int64_t)Q * ns + id], r_own - M(cz(Q)) * g);
    return S::template dec<Q>(fin[(int64_t)opp(Q) * ns + i], r_own);
}

// Known-sum of Eq. (inlet) on shifted values: K' = K - 1 (the weights of the
// listed distributions sum to exactly 1).
template <class M>
__device__ __forceinline__ M inlet_known(const M* d) {
    return d[0] + d[1] + d[2] + d[3] + d[4] + d[7] + d[8] + d[9] + d[10] +
           M(2) * (d[6] + d[12] + d[13] + d[16] + d[17]);
}
// Mirror for the outlet: sum over xi_z = 0 plus twice xi_z = +1, minus 1.
template <class M>
__device__ __forceinline__ M outlet_known(const M* d) {
    return d[0] + d[1] + d[2] + d[3] + d[4] + d[7] + d[8] + d[9] + d[10] +
           M(2) * (d[5] + d[11] + d[14] + d[15] + d[18]);
}

// Appendix B, Hecht-Harting closure at a z-inlet with u_x = u_y = 0:
// f5 = f6 + u_z/3, f11 = f12 + u_z/6 - N_x, f14 = f13 + u_z/6 + N_x,
// f15 = f16 + u_z/6 - N_y, f18 = f17 + u_z/6 + N_y (rho0 = 1); pairs share a
// weight so the same relations hold for d.
template <class M>
__device__ __forceinline__ void close_inlet(M* d, M uz) {
    const M nx = M(0.5) * (d[1] + d[7] + d[9] - d[2] - d[10] - d[8]);
    const M ny = M(0.5) * (d[3] + d[7] + d[10] - d[4] - d[9] - d[8]);
    const M u3 = uz * M(1.0 / 3.0), u6 = uz * M(1.0 / 6.0);
    d[5] = d[6] + u3;
    d[11] = d[12] + u6 - nx;
    d[14] = d[13] + u6 + nx;
    d[15] = d[16] + u6 - ny;
    d[18] = d[17] + u6 + ny;
}
// The same relations solved for the xi_z = -1 members at a z-outlet.
template <class M>
__device__ __forceinline__ void close_outlet(M* d, M uz) {
    const M nx = M(0.5) * (d[1] + d[7] + d[9] - d[2] - d[10] - d[8]);
    const M ny = M(0.5) * (d[3] + d[7] + d[10] - d[4] - d[9] - d[8]);
    const M u3 = uz * M(1.0 / 3.0), u6 = uz * M(1.0 / 6.0);
    d[6] = d[5] - u3;
    d[12] = d[11] - u6 + nx;
    d[13] = d[14] - u6 - nx;
    d[16] = d[15] - u6 + ny;
    d[17] = d[18] - u6 - ny;
}

// Collision on shifted values.  Appendix A's MRT with the paper's rates equals
// the two-relaxation-time update
//   f'_q = f_q - s+ (f+_q - feq+_q) - s- (f-_q - feq-_q)
// with f+- = (f_q +- f_opp)/2, s+ = 1/tau, s- = 8(2 - s+)/(8 - s+); BGK is
// s+ = s- = 1/tau.  feq_q - w_q = w_q (drho + 3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u)
// with u = j (rho0 = 1).
template <class M, int A>
__device__ __forceinline__ void relax_pair(M* d, M drho, M ux, M uy, M uz, M uu15, M sp, M sm) {
    constexpr int B = opp(A);
    const M xu = M(cx(A)) * ux + M(cy(A)) * uy + M(cz(A)) * uz;
    const M w = M(wq(A));
    const M ep = w * (drho + M(4.5) * xu * xu - uu15);
    const M em = w * M(3) * xu;
    const M dp = sp * (M(0.5) * (d[A] + d[B]) - ep);
    const M dm = sm * (M(0.5) * (d[A] - d[B]) - em);
    d[A] = d[A] - dp - dm;
    d[B] = d[B] - dp + dm;
}

template <class M>
__device__ __forceinline__ void moments(const M* d, M& drho, M& jx, M& jy, M& jz) {
    drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) +
           ((d[8] + d[9]) + (d[10] + d[11])) + ((d[12] + d[13]) + (d[14] + d[15])) +
           ((d[16] + d[17]) + d[18]);
    jx = (d[1] - d[2]) + (d[7] - d[8]) + (d[9] - d[10]) + (d[11] - d[12]) + (d[13] - d[14]);
    jy = (d[3] - d[4]) + (d[7] - d[8]) + (d[10] - d[9]) + (d[15] - d[16]) + (d[17] - d[18]);
    jz = (d[5] - d[6]) + (d[11] - d[12]) + (d[14] - d[13]) + (d[15] - d[16]) + (d[18] - d[17]);
}

template <class M>
__device__ __forceinline__ void collide(M* d, M sp, M sm) {
    M drho, ux, uy, uz;
    moments(d, drho, ux, uy, uz);
    const M uu15 = M(1.5) * (ux * ux + uy * uy + uz * uz);
    d[0] = d[0] - sp * (d[0] - M(wq(0)) * (drho - uu15));
    relax_pair<M, 1>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 3>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 5>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 7>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 9>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 11>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 13>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 15>(d, drho, ux, uy, uz, uu15, sp, sm);
    relax_pair<M, 17>(d, drho, ux, uy, uz, uu15, sp, sm);
}

}  // namespace lbm
