// Learned warm start: a 3-D convolutional U-Net that predicts the steady
// velocity field u / u_D of a pore geometry, trained on steady states this
// library computes, with its own CUDA forward, backward and Adam kernels.  The
// 3x3x3 convolutions run on the tcgen05 tensor cores: BF16 weights and
// activations, FP32 accumulation in tensor memory.
//
// Architecture (L levels, c_l = base * 2^l channels; every side divisible by
// 2^(L-1)):
//   E0a = relu(conv(X)), E0b = relu(conv(E0a))                      level 0
//   Ela = relu(conv(pool(E(l-1)b))), Elb = relu(conv(Ela))           l = 1 .. L-1
//   Dla = relu(conv(up(D(l+1)b))), Sl = Dla + Elb,                   l = L-2 .. 0
//   Dlb = relu(conv(Sl))                        (D(L-1)b = E(L-1)b)
//   Y   = conv(D0b) * X          (4 channels: u / u_D and G = -dp/dz / (nu u_D);
//                                 X = pore indicator)
// conv = 3x3x3 cross-correlation, zero padding, bias; pool = 2x2x2 mean;
// up = nearest 2x.  Loss = masked mean squared error over the entries that
// have a target (a NaN target entry has none).
// Parameters (FP32 master copy, Adam state) per layer: W[co][27][ci] (taps dz,
// dy, dx in -1..1, then the input channel) then b[co].
//
// Activation layout: BF16, channels last, with a one-voxel zero border:
// [B][Z+2][Y+2][X+2][C], C in {32, 64, 128, 256} (the 1-channel input and the
// 4-channel output are zero-padded to 32 channels).  In this layout a 3x3x3
// tap is a constant row offset, so the implicit-GEMM operand of tap t for the
// 128 output rows r0 .. r0+127 is the contiguous row range r0 + off(t): one
// TMA box.  Outputs on border rows are computed and discarded (written 0).
//
//   forward / data gradient (k_conv):  D[128 rows x Cout] = sum_t A_t[128 x Cin] W_t[Cin x Cout]
//     A: activation rows (K-major), B: weights [Cout][27*Cin] (K-major); K
//     streamed through a TMA -> shared memory -> tcgen05 pipeline in chunks
//     of 64 (or 32) channels of one tap.
//   weight gradient (k_wgrad):  D[(tap, ci) x co] = sum_rows act[r + off(tap)][ci] g[r][co]
//     A: 128 (tap, channel) pairs of shifted activation rows (MN-major),
//     B: output-gradient rows (MN-major); split over rows, FP32 atomics.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "tc_util.cuh"

typedef __nv_bfloat16 bf16;

namespace wsn {
namespace {

constexpr int kThreads = 192;  // warp 0: TMA, warp 1: MMA + TMEM, warps 2-5: epilogue
constexpr int kRows = 128;     // output rows per tile (MMA M)
constexpr int kOut = 4;        // network output channels: u / u_D (3), pressure gradient G

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int pow2_at_least(int v) {
    int p = 32;
    while (p < v) p *= 2;
    return p;
}

// ------------------------------------------------------------ geometry ---
struct PGeo {   // padded volume of B samples
    int B, X, Y, Z;
    __host__ __device__ int xp() const { return X + 2; }
    __host__ __device__ int64_t plane() const { return (int64_t)(Y + 2) * (X + 2); }
    __host__ __device__ int64_t per_sample() const { return (int64_t)(Z + 2) * plane(); }
    __host__ __device__ int64_t rows() const { return (int64_t)B * per_sample(); }
    __host__ __device__ int64_t row(int b, int z, int y, int x) const {  // interior coordinates
        return (int64_t)b * per_sample() + (int64_t)(z + 1) * plane() + (int64_t)(y + 1) * xp() + (x + 1);
    }
};

// interior coordinates of padded row r; false on a border row
__device__ __forceinline__ bool interior(const PGeo& g, int64_t r, int& b, int& z, int& y, int& x) {
    const int64_t xp = g.X + 2, yp = g.Y + 2, zp = g.Z + 2;
    int64_t t = r / xp;
    x = (int)(r - t * xp) - 1;
    int64_t t2 = t / yp;
    y = (int)(t - t2 * yp) - 1;
    int64_t t3 = t2 / zp;
    z = (int)(t2 - t3 * zp) - 1;
    b = (int)t3;
    return x >= 0 && x < g.X && y >= 0 && y < g.Y && z >= 0 && z < g.Z;
}

__device__ __forceinline__ int64_t tap_offset(int t, int64_t plane, int xp) {
    return (int64_t)(t / 9 - 1) * plane + (int64_t)((t / 3) % 3 - 1) * xp + (t % 3 - 1);
}

// 8 bf16 <-> 8 floats
__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 p = __bfloat1622float2(h[i]);
        f[2 * i] = p.x;
        f[2 * i + 1] = p.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

// ---------------------------------------------- forward / data gradient ---
template <int CIN, int COUT>
struct ConvCfg {
    static constexpr int AW = cmin(CIN, 64);            // channels per K chunk
    static constexpr int KSUB = CIN / AW;               // chunks per tap
    // FUSE (narrow outputs): one stage holds the 130 rows r0 - 1 .. r0 + 128 of
    // one (dz, dy) row window (one swizzled TMA box) and the weights of its three
    // dx taps; the three taps' A operands are the same window started one row
    // (AW * 2 bytes) apart, so a tile loads its input rows 9 times instead of 27.
    // Wide outputs keep one tap per stage (128 rows): their weights, not the
    // activations, dominate the bytes.  Measured on the 32 -> 32 layer, 8 x 64^3
    // voxels, per forward launch: 0.474 ms one tap per stage, 0.390 ms with the
    // window as four unswizzled 8-channel planes, 0.318 ms as one swizzled box,
    // 0.311 ms with the three taps' weights as one box of the tap-major copy;
    // slower: a persistent form with two TMEM accumulators (0.416 ms), weights
    // kept resident in shared memory (0.557 ms one tile per CTA, 0.458 ms
    // persistent).
    static constexpr bool FUSE = COUT <= 64;
    static constexpr int NITER = (FUSE ? 9 : 27) * KSUB;
    static constexpr int HALO = kRows + 2;
    static constexpr uint32_t A_BYTES = FUSE ? (HALO * AW * 2 + 1023) / 1024 * 1024 : kRows * AW * 2;
    static constexpr uint32_t A_TX = FUSE ? HALO * AW * 2 : A_BYTES;  // bytes the TMA delivers
    static constexpr uint32_t B_TAP = COUT * AW * 2;
    static constexpr uint32_t B_BYTES = (FUSE ? 3 : 1) * B_TAP;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t STAGE_TX = A_TX + B_BYTES;
    static constexpr int STAGES = 4 * STAGE <= 100 * 1024 ? cmin(8, (int)((96 * 1024) / STAGE))
                                                          : cmin(6, (int)((196 * 1024) / STAGE));
    static constexpr uint32_t A_REGION = (STAGES * A_BYTES + 1023) / 1024 * 1024;  // B stays 1024-aligned
    static constexpr uint32_t SWZ = AW == 64 ? 2u : 4u;  // 128-byte or 64-byte swizzle (B; A when not FUSE)
    static constexpr uint32_t SBO = 8 * AW * 2;          // 8-row core-matrix group stride (swizzled)
    static constexpr uint32_t COLS = COUT;
    static constexpr size_t SMEM = 1024 + (size_t)A_REGION + (size_t)STAGES * B_BYTES + 256;
};

struct ConvEpi {
    const float* bias;          // [COUT] or null
    int relu;
    bf16* out;                  // v (may be null)
    const bf16* add;            // out_add = v + add
    bf16* out_add;
    const bf16* mask;           // out_mask = v * (mask > 0)
    bf16* out_mask;
    float* y;                   // output layer: y[b][c][z][y][x] = v * pore, c < kOut
    const bf16* xin;            // pore indicator rows (channel 0 of a 32-channel tensor)
    int* err;
    PGeo g;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
k_conv(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, ConvEpi e) {
    using K = ConvCfg<CIN, COUT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + K::A_REGION;
    uint64_t* full = (uint64_t*)(sB + K::STAGES * K::B_BYTES);
    uint64_t* empty = full + K::STAGES;
    uint64_t* accb = empty + K::STAGES;
    uint32_t* tslot = (uint32_t*)(accb + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    if (threadIdx.x == 0) {
        for (int s = 0; s < K::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accb, 1);
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tslot, K::COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int64_t plane = e.g.plane();
    const int xp = e.g.xp();
    if (warp == 0) {
        if (lane == 0) {
            for (int j = 0; j < K::NITER; ++j) {
                const int s = j % K::STAGES, use = j / K::STAGES;
                if (use > 0 && !tc::mbar_wait(&empty[s], (use - 1) & 1, e.err)) break;
                const int w = j / K::KSUB, kc = j % K::KSUB;  // w: (dz, dy) window if FUSE, else the tap
                tc::mbar_expect_tx(&full[s], K::STAGE_TX);
                if constexpr (K::FUSE) {
                    // rows of taps (w, dx = -1..1): r0 + off(3 w + 1) - 1 .. + 129
                    const int row = (int)(r0 + tap_offset(3 * w + 1, plane, xp) - 1);
                    tc::tma_load_2d(sA + s * K::A_BYTES, &mA, &full[s], kc * K::AW, row);
                    // taps 3 w .. 3 w + 2 of the tap-major weights: one box of 3 COUT rows
                    tc::tma_load_2d(sB + s * K::B_BYTES, &mB, &full[s], kc * K::AW, 3 * w * COUT);
                } else {
                    tc::tma_load_2d(sA + s * K::A_BYTES, &mA, &full[s], kc * K::AW,
                                    (int)(r0 + tap_offset(w, plane, xp)));
                    tc::tma_load_2d(sB + s * K::B_BYTES, &mB, &full[s], w * CIN + kc * K::AW, 0);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(kRows, COUT, false, false);
            for (int j = 0; j < K::NITER; ++j) {
                const int s = j % K::STAGES, use = j / K::STAGES;
                if (!tc::mbar_wait(&full[s], use & 1, e.err)) break;
                tc::fence_after_sync();
                const uint32_t a = tc::su32(sA + s * K::A_BYTES), b = tc::su32(sB + s * K::B_BYTES);
                if constexpr (K::FUSE) {
                    // the swizzled window started dx rows in (the swizzle follows the
                    // absolute shared-memory address, so a row offset needs no base offset)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                        for (int k = 0; k < K::AW / 16; ++k)
                            tc::mma_bf16(tmem, tc::smem_desc(a + dx * K::AW * 2 + k * 32, 16, K::SBO, K::SWZ),
                                         tc::smem_desc(b + dx * K::B_TAP + k * 32, 16, K::SBO, K::SWZ), idesc,
                                         (j | dx | k) != 0);
                } else {
#pragma unroll
                    for (int k = 0; k < K::AW / 16; ++k)
                        tc::mma_bf16(tmem, tc::smem_desc(a + k * 32, 16, K::SBO, K::SWZ),
                                     tc::smem_desc(b + k * 32, 16, K::SBO, K::SWZ), idesc, (j | k) != 0);
                }
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(accb);
        }
    } else {
        const int q = warp & 3;  // TMEM lane quadrant this warp may read
        const bool ok = tc::mbar_wait(accb, 0, e.err);
        tc::fence_after_sync();
        const int64_t r = r0 + q * 32 + lane;
        int b = 0, z = 0, y = 0, x = 0;
        const bool in_range = r < e.g.rows();
        const bool inner = in_range && interior(e.g, r, b, z, y, x);
#pragma unroll 1
        for (int c0 = 0; c0 < COUT; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + c0, v);
            if (!ok || !in_range) continue;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float w = v[i] + (e.bias ? __ldg(e.bias + c0 + i) : 0.f);
                if (e.relu) w = fmaxf(w, 0.f);
                v[i] = inner ? w : 0.f;
            }
            const int64_t o = r * COUT + c0;
            if (e.out) {
                uint4* d = reinterpret_cast<uint4*>(e.out + o);
#pragma unroll
                for (int k = 0; k < 4; ++k) d[k] = pack8(v + 8 * k);
            }
            if (e.out_add) {
                const uint4* a = reinterpret_cast<const uint4*>(e.add + o);
                uint4* d = reinterpret_cast<uint4*>(e.out_add + o);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float f[8];
                    unpack8(a[k], f);
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[i] += v[8 * k + i];
                    d[k] = pack8(f);
                }
            }
            if (e.out_mask) {
                const uint4* m = reinterpret_cast<const uint4*>(e.mask + o);
                uint4* d = reinterpret_cast<uint4*>(e.out_mask + o);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float f[8];
                    unpack8(m[k], f);
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[i] = f[i] > 0.f ? v[8 * k + i] : 0.f;
                    d[k] = pack8(f);
                }
            }
            if (e.y && c0 == 0 && inner) {
                const float pore = __bfloat162float(e.xin[r * 32]) > 0.f ? 1.f : 0.f;
                const int64_t n = (int64_t)e.g.Z * e.g.Y * e.g.X;
                const int64_t o3 = ((int64_t)z * e.g.Y + y) * e.g.X + x;
#pragma unroll
                for (int c = 0; c < kOut; ++c) e.y[((int64_t)b * kOut + c) * n + o3] = v[c] * pore;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, K::COLS);
    }
}

// ----------------------------------------------------- weight gradient ---
template <int CIN, int COUT>
struct WgCfg {
    static constexpr int AW = cmin(CIN, 64);
    static constexpr int BW = cmin(COUT, 64);
    static constexpr int ABLK = 128 / AW;                 // MN blocks of A (128 (tap, ci) pairs)
    static constexpr int BBLK = COUT / BW;
    static constexpr uint32_t A_BLK = kRows * AW * 2;
    static constexpr uint32_t B_BLK = kRows * BW * 2;
    static constexpr uint32_t A_BYTES = ABLK * A_BLK;     // 32 KB
    static constexpr uint32_t B_BYTES = BBLK * B_BLK;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = cmin(4, (int)((200 * 1024) / STAGE));
    static constexpr int NG = (27 * CIN + 127) / 128;     // groups of 128 (tap, ci) pairs
    static constexpr int GPC = cmin(NG, 512 / COUT);      // groups accumulated per CTA
    static constexpr int COLS = pow2_at_least(GPC * COUT);
    static constexpr uint32_t ASWZ = AW == 64 ? 2u : 4u, BSWZ = BW == 64 ? 2u : 4u;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
};

struct WgArgs {
    float* gw;           // FP32 [cout_real][27][cin_real], accumulated
    int cin_real, cout_real;
    int64_t nchunks;     // row chunks of 128 in the volume
    int* err;
    PGeo g;
    // Deterministic form: each row split stores its partial sums in
    // part[split][cout_real][27][cin_real] (part_cap floats available) and a
    // second kernel adds them to gw in split order; null: FP32 atomics into gw.
    float* part;
    int64_t part_cap;
};

// Row splits of a weight-gradient launch: enough CTAs for two per SM over the
// groups of 128 (tap, c_in) pairs, at most one per 128-row chunk.
inline int64_t wgrad_splits(int cin, int cout, int64_t rows, int n_sm) {
    const int ng = (27 * cin + 127) / 128;
    const int gpc = std::min(ng, 512 / cout);
    const int gsets = (ng + gpc - 1) / gpc;
    const int64_t want = std::max<int64_t>(1, (2 * (int64_t)n_sm + gsets - 1) / gsets);
    return std::min<int64_t>(want, (rows + kRows - 1) / kRows);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
k_wgrad(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mG, WgArgs a) {
    using K = WgCfg<CIN, COUT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + K::STAGES * K::A_BYTES;
    uint64_t* full = (uint64_t*)(sB + K::STAGES * K::B_BYTES);
    uint64_t* empty = full + K::STAGES;
    uint64_t* accb = empty + K::STAGES;
    uint32_t* tslot = (uint32_t*)(accb + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g0 = blockIdx.y * K::GPC;
    const int ng = cmin(K::GPC, K::NG - g0);
    const int64_t c_begin = a.nchunks * blockIdx.x / gridDim.x;
    const int64_t c_end = a.nchunks * (blockIdx.x + 1) / gridDim.x;
    const int64_t n_iter = (c_end - c_begin) * ng;
    if (threadIdx.x == 0) {
        for (int s = 0; s < K::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accb, 1);
        tc::mbar_init_fence();
    }
    if (warp == 1) tc::tmem_alloc(tslot, K::COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int64_t plane = a.g.plane();
    const int xp = a.g.xp();
    if (warp == 0) {
        if (lane == 0) {
            for (int64_t j = 0; j < n_iter; ++j) {
                const int s = (int)(j % K::STAGES);
                const int64_t use = j / K::STAGES;
                if (use > 0 && !tc::mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), a.err)) break;
                const int64_t r0 = (c_begin + j / ng) * kRows;
                const int grp = g0 + (int)(j % ng);
                tc::mbar_expect_tx(&full[s], K::STAGE);
#pragma unroll
                for (int bk = 0; bk < K::ABLK; ++bk) {
                    const int p0 = grp * 128 + bk * K::AW;
                    const int tap = cmin(p0 / CIN, 26);  // pairs past the last tap load tap 26 (ignored)
                    tc::tma_load_2d(sA + s * K::A_BYTES + bk * K::A_BLK, &mA, &full[s], p0 % CIN,
                                    (int)(r0 + tap_offset(tap, plane, xp)));
                }
#pragma unroll
                for (int bk = 0; bk < K::BBLK; ++bk)
                    tc::tma_load_2d(sB + s * K::B_BYTES + bk * K::B_BLK, &mG, &full[s], bk * K::BW, (int)r0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(kRows, COUT, true, true);
            for (int64_t j = 0; j < n_iter; ++j) {
                const int s = (int)(j % K::STAGES);
                const int64_t use = j / K::STAGES;
                if (!tc::mbar_wait(&full[s], (uint32_t)(use & 1), a.err)) break;
                tc::fence_after_sync();
                const int gl = (int)(j % ng);
                const bool first = j < ng;  // first row chunk of this group
                const uint32_t aa = tc::su32(sA + s * K::A_BYTES), bb = tc::su32(sB + s * K::B_BYTES);
#pragma unroll
                for (int k = 0; k < 8; ++k)  // K = 16 rows per MMA
                    tc::mma_bf16(tmem + gl * COUT,
                                 tc::smem_desc(aa + k * 16 * K::AW * 2, K::A_BLK, 8 * K::AW * 2, K::ASWZ),
                                 tc::smem_desc(bb + k * 16 * K::BW * 2, K::B_BLK, 8 * K::BW * 2, K::BSWZ), idesc,
                                 !(first && k == 0));
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(accb);
        }
    } else {
        const int q = warp & 3;
        const bool ok = tc::mbar_wait(accb, 0, a.err) && n_iter > 0;
        tc::fence_after_sync();
#pragma unroll 1
        for (int gl = 0; gl < ng; ++gl) {
            const int p = (g0 + gl) * 128 + q * 32 + lane;
            const int tap = p / CIN, ci = p % CIN;
            const bool valid = ok && tap < 27 && ci < a.cin_real;
#pragma unroll 1
            for (int c0 = 0; c0 < COUT; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + gl * COUT + c0, v);
                if (!valid) continue;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int co = c0 + i;
                    if (co >= a.cout_real) continue;
                    const int64_t w = ((int64_t)co * 27 + tap) * a.cin_real + ci;
                    if (a.part) a.part[(int64_t)blockIdx.x * ((int64_t)a.cout_real * 27 * a.cin_real) + w] = v[i];
                    else atomicAdd(a.gw + w, v[i]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, K::COLS);
    }
}

// ------------------------------------------------- elementwise kernels ---
inline unsigned gs_blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32); }

// X32[row] = (pore, 0, ..., 0) on interior rows; masks uint8 [B][Z][Y][X], 1 = solid
__global__ void k_x32(const uint8_t* __restrict__ mask, bf16* __restrict__ x32, PGeo g) {
    const int64_t n = (int64_t)g.B * g.Z * g.Y * g.X;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % g.X);
        const int64_t t = k / g.X;
        const int y = (int)(t % g.Y), z = (int)((t / g.Y) % g.Z), b = (int)(t / ((int64_t)g.Y * g.Z));
        float f[8] = {mask[k] ? 0.f : 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4* d = reinterpret_cast<uint4*>(x32 + g.row(b, z, y, x) * 32);
        d[0] = pack8(f);
        f[0] = 0.f;
        const uint4 zero = pack8(f);
        d[1] = zero;
        d[2] = zero;
        d[3] = zero;
    }
}

// coarse[v][c] = mean of the 8 fine children; one thread per (coarse voxel, 8 channels)
__global__ void k_pool(const bf16* __restrict__ fine, bf16* __restrict__ coarse, PGeo gc, PGeo gf, int C) {
    const int cg = C / 8;
    const int64_t n = (int64_t)gc.B * gc.Z * gc.Y * gc.X * cg;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int c8 = (int)(k % cg);
        int64_t t = k / cg;
        const int x = (int)(t % gc.X);
        t /= gc.X;
        const int y = (int)(t % gc.Y);
        t /= gc.Y;
        const int z = (int)(t % gc.Z), b = (int)(t / gc.Z);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int d = 0; d < 8; ++d) {
            float f[8];
            unpack8(*reinterpret_cast<const uint4*>(
                        fine + gf.row(b, 2 * z + (d >> 2), 2 * y + ((d >> 1) & 1), 2 * x + (d & 1)) * C + c8 * 8),
                    f);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] += f[i];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] *= 0.125f;
        *reinterpret_cast<uint4*>(coarse + gc.row(b, z, y, x) * C + c8 * 8) = pack8(acc);
    }
}

// fine[v][c] = coarse[parent(v)][c]
__global__ void k_up(const bf16* __restrict__ coarse, bf16* __restrict__ fine, PGeo gf, PGeo gc, int C) {
    const int cg = C / 8;
    const int64_t n = (int64_t)gf.B * gf.Z * gf.Y * gf.X * cg;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int c8 = (int)(k % cg);
        int64_t t = k / cg;
        const int x = (int)(t % gf.X);
        t /= gf.X;
        const int y = (int)(t % gf.Y);
        t /= gf.Y;
        const int z = (int)(t % gf.Z), b = (int)(t / gf.Z);
        *reinterpret_cast<uint4*>(fine + gf.row(b, z, y, x) * C + c8 * 8) =
            *reinterpret_cast<const uint4*>(coarse + gc.row(b, z / 2, y / 2, x / 2) * C + c8 * 8);
    }
}

// out[v][c] = (sum of the 8 children of gfine) * (act[v][c] > 0)   (adjoint of up, then relu')
__global__ void k_up_bwd_mask(const bf16* __restrict__ gfine, const bf16* __restrict__ act, bf16* __restrict__ out,
                              PGeo gc, PGeo gf, int C) {
    const int cg = C / 8;
    const int64_t n = (int64_t)gc.B * gc.Z * gc.Y * gc.X * cg;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int c8 = (int)(k % cg);
        int64_t t = k / cg;
        const int x = (int)(t % gc.X);
        t /= gc.X;
        const int y = (int)(t % gc.Y);
        t /= gc.Y;
        const int z = (int)(t % gc.Z), b = (int)(t / gc.Z);
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int d = 0; d < 8; ++d) {
            float f[8];
            unpack8(*reinterpret_cast<const uint4*>(
                        gfine + gf.row(b, 2 * z + (d >> 2), 2 * y + ((d >> 1) & 1), 2 * x + (d & 1)) * C + c8 * 8),
                    f);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] += f[i];
        }
        const int64_t o = gc.row(b, z, y, x) * C + c8 * 8;
        float m[8];
        unpack8(*reinterpret_cast<const uint4*>(act + o), m);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = m[i] > 0.f ? acc[i] : 0.f;
        *reinterpret_cast<uint4*>(out + o) = pack8(acc);
    }
}

// out[v][c] = (gacc[v][c] + gcoarse[parent(v)][c] / 8) * (act[v][c] > 0)   (adjoint of pool + skip, then relu')
__global__ void k_pool_bwd_add_mask(const bf16* __restrict__ gcoarse, const bf16* __restrict__ gacc,
                                    const bf16* __restrict__ act, bf16* __restrict__ out, PGeo gf, PGeo gc, int C) {
    const int cg = C / 8;
    const int64_t n = (int64_t)gf.B * gf.Z * gf.Y * gf.X * cg;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int c8 = (int)(k % cg);
        int64_t t = k / cg;
        const int x = (int)(t % gf.X);
        t /= gf.X;
        const int y = (int)(t % gf.Y);
        t /= gf.Y;
        const int z = (int)(t % gf.Z), b = (int)(t / gf.Z);
        const int64_t o = gf.row(b, z, y, x) * C + c8 * 8;
        float f[8], s[8], m[8];
        unpack8(*reinterpret_cast<const uint4*>(gcoarse + gc.row(b, z / 2, y / 2, x / 2) * C + c8 * 8), f);
        unpack8(*reinterpret_cast<const uint4*>(gacc + o), s);
        unpack8(*reinterpret_cast<const uint4*>(act + o), m);
#pragma unroll
        for (int i = 0; i < 8; ++i) f[i] = m[i] > 0.f ? s[i] + 0.125f * f[i] : 0.f;
        *reinterpret_cast<uint4*>(out + o) = pack8(f);
    }
}

// masked MSE over interior voxels: gz[row] = (2 inv (Y - T) pore for c < kOut with a target, 0 else),
// loss += inv sum (Y - T)^2 pore; a NaN target entry has no target
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, const bf16* __restrict__ x32,
                      bf16* __restrict__ gz, PGeo g, double inv, double* loss) {
    __shared__ double sh[32];
    const int64_t n = (int64_t)g.B * g.Z * g.Y * g.X;
    const int64_t N = (int64_t)g.Z * g.Y * g.X;
    double s = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % g.X);
        const int64_t t = k / g.X;
        const int y = (int)(t % g.Y), z = (int)((t / g.Y) % g.Z), b = (int)(t / ((int64_t)g.Y * g.Z));
        const int64_t r = g.row(b, z, y, x);
        const float pore = __bfloat162float(x32[r * 32]) > 0.f ? 1.f : 0.f;
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int64_t o = (int64_t)b * kOut * N + k - (int64_t)b * N;
        for (int c = 0; c < kOut; ++c) {
            const float t = T[o + c * N];
            const float d = t == t ? (Y[o + c * N] - t) * pore : 0.f;
            f[c] = (float)(2.0 * inv) * d;
            s += (double)d * d;
        }
        uint4* d = reinterpret_cast<uint4*>(gz + r * 32);
        d[0] = pack8(f);
        for (int c = 0; c < kOut; ++c) f[c] = 0.f;
        const uint4 zero = pack8(f);
        d[1] = zero;
        d[2] = zero;
        d[3] = zero;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(loss, s * inv);
    }
}

// gw[w] += sum over k of part[k][w], k in order (the deterministic finish of
// the weight- and bias-gradient kernels)
__global__ void k_split_sum(const float* __restrict__ part, int64_t splits, int64_t nw, float* __restrict__ gw) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int64_t k = 0; k < splits; ++k) s += part[k * nw + w];
        gw[w] += s;
    }
}

// gb[c] += sum over rows of G[row][c], c < creal; block of 256 threads, C / 8 channel groups.
// With `part`, block b stores its sums in part[b][c] instead (no atomics).
__global__ void k_bias_grad(const bf16* __restrict__ G, int64_t rows, int C, int creal, float* __restrict__ gb,
                            float* __restrict__ part) {
    __shared__ float sh[256][8];
    const int cg = C / 8;
    const int lanes = 256 / cg;  // threads per channel group
    const int c8 = threadIdx.x % cg, sub = threadIdx.x / cg;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (sub < lanes)
        for (int64_t r = (int64_t)blockIdx.x * lanes + sub; r < rows; r += (int64_t)gridDim.x * lanes) {
            float f[8];
            unpack8(*reinterpret_cast<const uint4*>(G + r * C + c8 * 8), f);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] += f[i];
        }
#pragma unroll
    for (int i = 0; i < 8; ++i) sh[threadIdx.x][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < cg) {
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int u = 0; u < lanes; ++u)
#pragma unroll
            for (int i = 0; i < 8; ++i) s[i] += sh[u * cg + threadIdx.x][i];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = threadIdx.x * 8 + i;
            if (c >= creal) continue;
            if (part) part[(int64_t)blockIdx.x * creal + c] = s[i];
            else atomicAdd(gb + c, s[i]);
        }
    }
}

struct LayerDesc {
    int cout, cin, cout_p, cin_p;
    int64_t woff, boff;      // into the FP32 parameter vector
    int64_t wf, wb, bp;      // into the BF16 weight store / padded bias store
    int64_t wft, wbt;        // the same weights tap-major: [t][cout][cin] and [t][cin][cout]
};

// BF16 forward weights wf[co][t][ci], data-gradient weights wb[ci][t][co] =
// W[co][26 - t][ci] and padded biases, zero in the padding channels.
__global__ void k_pack(const float* __restrict__ p, const LayerDesc* __restrict__ L, int nl, bf16* __restrict__ wst,
                       float* __restrict__ bst) {
    const LayerDesc d = L[blockIdx.y];
    const int64_t n = (int64_t)d.cout_p * 27 * d.cin_p;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(k % d.cin_p), t = (int)((k / d.cin_p) % 27), co = (int)(k / (27 * d.cin_p));
        const bool real = co < d.cout && ci < d.cin;
        const bf16 v = __float2bfloat16_rn(real ? p[d.woff + ((int64_t)co * 27 + t) * d.cin + ci] : 0.f);
        wst[d.wf + k] = v;
        wst[d.wb + ((int64_t)ci * 27 + (26 - t)) * d.cout_p + co] = v;
        wst[d.wft + ((int64_t)t * d.cout_p + co) * d.cin_p + ci] = v;
        wst[d.wbt + ((int64_t)(26 - t) * d.cin_p + ci) * d.cout_p + co] = v;
    }
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < d.cout_p; c += blockDim.x) bst[d.bp + c] = c < d.cout ? p[d.boff + c] : 0.f;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// ------------------------------------------------------- host helpers ---
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t get_encode() {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// 2-D map of a [rows][C] BF16 tensor with a box of (box_c channels, box_r rows)
cudaError_t make_map(CUtensorMap* m, const void* ptr, int C, int64_t rows, int box_c, int box_r) {
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)C * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_c, (cuuint32_t)box_r};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapSwizzle sw = box_c * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : box_c * 2 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE;
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// w: weights [COUT][27][CIN]; wt: the same tap-major, [27][COUT][CIN] (the
// fused layers load the three dx taps of a tap row as one box from it)
template <int CIN, int COUT>
cudaError_t conv_t(const bf16* in, const bf16* w, const bf16* wt, const ConvEpi& epi, cudaStream_t st) {
    using K = ConvCfg<CIN, COUT>;
    cudaError_t e0 = cudaFuncSetAttribute(k_conv<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
    if (e0 != cudaSuccess) return e0;
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, in, CIN, epi.g.rows(), K::AW, K::FUSE ? K::HALO : kRows);
    if (e == cudaSuccess)
        e = K::FUSE ? make_map(&mb, wt, CIN, 27 * COUT, K::AW, 3 * COUT) : make_map(&mb, w, 27 * CIN, COUT, K::AW, COUT);
    if (e != cudaSuccess) return e;
    const unsigned tiles = (unsigned)((epi.g.rows() + kRows - 1) / kRows);
    k_conv<CIN, COUT><<<tiles, kThreads, K::SMEM, st>>>(ma, mb, epi);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad_t(const bf16* act, const bf16* gout, const WgArgs& a0, cudaStream_t st, int n_sm) {
    using K = WgCfg<CIN, COUT>;
    cudaError_t e0 = cudaFuncSetAttribute(k_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
    if (e0 != cudaSuccess) return e0;
    CUtensorMap ma, mg;
    cudaError_t e = make_map(&ma, act, CIN, a0.g.rows(), K::AW, kRows);
    if (e == cudaSuccess) e = make_map(&mg, gout, COUT, a0.g.rows(), K::BW, kRows);
    if (e != cudaSuccess) return e;
    WgArgs a = a0;
    a.nchunks = (a.g.rows() + kRows - 1) / kRows;
    const int gsets = (K::NG + K::GPC - 1) / K::GPC;
    const unsigned splits = (unsigned)wgrad_splits(CIN, COUT, a.g.rows(), n_sm);
    const int64_t nw = (int64_t)a.cout_real * 27 * a.cin_real;
    if (a.part && (int64_t)splits * nw > a.part_cap) return cudaErrorInvalidValue;
    k_wgrad<CIN, COUT><<<dim3(splits, (unsigned)gsets), kThreads, K::SMEM, st>>>(ma, mg, a);
    if (a.part) k_split_sum<<<gs_blocks(nw), 256, 0, st>>>(a.part, splits, nw, a.gw);
    return cudaGetLastError();
}

#define WS_DISPATCH(FN, CIN, COUT, ...)                                      \
    switch (CIN * 1000 + COUT) {                                             \
        case 32032: return FN<32, 32>(__VA_ARGS__);                          \
        case 32064: return FN<32, 64>(__VA_ARGS__);                          \
        case 32128: return FN<32, 128>(__VA_ARGS__);                         \
        case 32256: return FN<32, 256>(__VA_ARGS__);                         \
        case 64032: return FN<64, 32>(__VA_ARGS__);                          \
        case 64064: return FN<64, 64>(__VA_ARGS__);                          \
        case 64128: return FN<64, 128>(__VA_ARGS__);                         \
        case 64256: return FN<64, 256>(__VA_ARGS__);                         \
        case 128032: return FN<128, 32>(__VA_ARGS__);                        \
        case 128064: return FN<128, 64>(__VA_ARGS__);                        \
        case 128128: return FN<128, 128>(__VA_ARGS__);                       \
        case 128256: return FN<128, 256>(__VA_ARGS__);                       \
        case 256032: return FN<256, 32>(__VA_ARGS__);                        \
        case 256064: return FN<256, 64>(__VA_ARGS__);                        \
        case 256128: return FN<256, 128>(__VA_ARGS__);                       \
        case 256256: return FN<256, 256>(__VA_ARGS__);                       \
        default: return cudaErrorInvalidValue;                               \
    }

cudaError_t conv(int cin, int cout, const bf16* in, const bf16* w, const bf16* wt, const ConvEpi& epi,
                 cudaStream_t st) {
    WS_DISPATCH(conv_t, cin, cout, in, w, wt, epi, st)
}
cudaError_t wgrad(int cin, int cout, const bf16* act, const bf16* gout, const WgArgs& a, cudaStream_t st, int n_sm) {
    WS_DISPATCH(wgrad_t, cin, cout, act, gout, a, st, n_sm)
}

bool chan_ok(int c) { return c == 32 || c == 64 || c == 128 || c == 256; }

}  // namespace
}  // namespace wsn

// ================================================================ network ===
struct lbm_wsnet {
    int device = 0;
    int n_sm = 152;
    int levels = 4, base = 32;
    std::vector<wsn::LayerDesc> L;      // host copy
    wsn::LayerDesc* d_L = nullptr;
    int64_t np = 0, nw = 0, nb = 0;     // FP32 parameters, BF16 weight elements, padded bias floats
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16* wst = nullptr;                // packed BF16 weights (forward and data-gradient layouts)
    float* bst = nullptr;               // padded biases
    double* d_loss = nullptr;
    int* d_err = nullptr;
    float* part = nullptr;              // per-split partial gradient sums (deterministic accumulation)
    int64_t part_cap = 0;               // floats
    int64_t adam_t = 0;
    bool packed = false;
    cudaStream_t stream = nullptr;
    // activation / gradient buffers of the current (batch, geometry)
    std::map<std::string, void*> buf;
    int gB = 0, gX = 0, gY = 0, gZ = 0;  // current batch and volume
    int capB = 0;                        // batch the buffers were allocated for
    std::string err;
    int status = LBM_OK;
};

namespace {

using wsn::PGeo;

int wfail(lbm_wsnet* n, int code, const char* fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    if (n) {
        n->err = b;
        if (code == LBM_ECUDA) n->status = LBM_ECUDA;
    }
    return code;
}
#define WS_CUDA(n, call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return wfail((n), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int wenter(lbm_wsnet* n) {
    if (!n) return LBM_EINVAL;
    if (n->status == LBM_ECUDA) return LBM_ECUDA;
    WS_CUDA(n, cudaSetDevice(n->device));
    return LBM_OK;
}

void free_buffers(lbm_wsnet* n) {
    for (auto& kv : n->buf) cudaFree(kv.second);
    n->buf.clear();
    n->gB = n->gX = n->gY = n->gZ = n->capB = 0;
}

PGeo level_geo(const lbm_wsnet* n, int l) {
    return PGeo{n->gB, n->gX >> l, n->gY >> l, n->gZ >> l};
}

int chans(const lbm_wsnet* n, int l) { return n->base << l; }

// Make sure the buffers for (B, X, Y, Z) exist (with the gradient buffers if
// `grads`); every buffer starts zeroed so its border rows are zero (no kernel
// writes a non-zero value there).
int ensure_buffers(lbm_wsnet* n, int B, int X, int Y, int Z, bool grads) {
    // a batch no larger than the allocated one reuses the buffers (the rows of
    // the samples past B are left alone, so every border row stays zero)
    const bool fits = n->gX == X && n->gY == Y && n->gZ == Z && B <= n->capB && !n->buf.empty();
    if (fits && (!grads || n->buf.count("gZ"))) {
        n->gB = B;
        return LBM_OK;
    }
    WS_CUDA(n, cudaStreamSynchronize(n->stream));
    if (!fits) {
        free_buffers(n);
        n->capB = B;
    }
    n->gB = n->capB;  // allocation sizes
    n->gX = X;
    n->gY = Y;
    n->gZ = Z;
    auto alloc = [&](const std::string& name, size_t bytes) -> int {
        if (n->buf.count(name)) return LBM_OK;
        void* d = nullptr;
        cudaError_t e = cudaMalloc(&d, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            free_buffers(n);
            return wfail(n, LBM_ENOMEM, "network buffer %s (%zu bytes): %s", name.c_str(), bytes,
                         cudaGetErrorString(e));
        }
        n->buf[name] = d;
        e = cudaMemsetAsync(d, 0, bytes, n->stream);
        if (e != cudaSuccess) return wfail(n, LBM_ECUDA, "memset: %s", cudaGetErrorString(e));
        return LBM_OK;
    };
    auto act = [&](const std::string& name, int l, int C) { return alloc(name, (size_t)level_geo(n, l).rows() * C * 2); };
    const int Lv = n->levels;
    int rc = LBM_OK;
    const int64_t vox = (int64_t)n->capB * X * Y * Z;
    if ((rc = act("X", 0, 32))) return rc;
    if ((rc = alloc("Y", (size_t)vox * wsn::kOut * 4))) return rc;
    if ((rc = alloc("M", (size_t)vox))) return rc;
    for (int l = 0; l < Lv; ++l) {
        const int C = chans(n, l);
        char s[32];
        auto nm = [&](const char* f) { snprintf(s, sizeof s, f, l); return std::string(s); };
        if ((rc = act(nm("E%da"), l, C)) || (rc = act(nm("E%db"), l, C))) return rc;
        if (l > 0 && (rc = act(nm("P%d"), l, chans(n, l - 1)))) return rc;
        if (l <= Lv - 2 && ((rc = act(nm("U%d"), l, chans(n, l + 1))) || (rc = act(nm("D%da"), l, C)) ||
                            (rc = act(nm("S%d"), l, C)) || (rc = act(nm("D%db"), l, C))))
            return rc;
        if (!grads) continue;
        if (l <= Lv - 2 && ((rc = act(nm("gskip%d"), l, C)) || (rc = act(nm("gU%d"), l, chans(n, l + 1)))))
            return rc;
        if ((rc = act(nm("gA%d"), l, C)) || (rc = act(nm("gB%d"), l, C))) return rc;
        if (l > 0 && (rc = act(nm("gP%d"), l, chans(n, l - 1)))) return rc;
    }
    if (grads) {
        if ((rc = alloc("T", (size_t)vox * wsn::kOut * 4))) return rc;
        if ((rc = act("gZ", 0, 32))) return rc;  // last: its presence marks the gradient buffers
    }
    n->gB = B;
    return LBM_OK;
}

bf16* B16(lbm_wsnet* n, const std::string& k) { return (bf16*)n->buf.at(k); }

int pack_weights(lbm_wsnet* n) {
    const int nl = (int)n->L.size();
    wsn::k_pack<<<dim3(64, (unsigned)nl), 256, 0, n->stream>>>(n->p, n->d_L, nl, n->wst, n->bst);
    WS_CUDA(n, cudaGetLastError());
    n->packed = true;
    return LBM_OK;
}

// conv layer k forward: out = act(W_k * in + b_k) with optional fused outputs
int fwd_layer(lbm_wsnet* n, int k, const bf16* in, int l, bool relu, bf16* out, const bf16* add, bf16* out_add,
              float* y = nullptr, const bf16* xin = nullptr) {
    const wsn::LayerDesc& d = n->L[k];
    wsn::ConvEpi e{};
    e.bias = n->bst + d.bp;
    e.relu = relu;
    e.out = out;
    e.add = add;
    e.out_add = out_add;
    e.y = y;
    e.xin = xin;
    e.err = n->d_err;
    e.g = level_geo(n, l);
    WS_CUDA(n, wsn::conv(d.cin_p, d.cout_p, in, n->wst + d.wf, n->wst + d.wft, e, n->stream));
    return LBM_OK;
}

// conv layer k data gradient: g_in = W_k^T * g_out; out = g_in, out_mask = g_in * (mask > 0)
int bwd_data(lbm_wsnet* n, int k, const bf16* gout, int l, bf16* out, const bf16* mask, bf16* out_mask) {
    const wsn::LayerDesc& d = n->L[k];
    wsn::ConvEpi e{};
    e.out = out;
    e.mask = mask;
    e.out_mask = out_mask;
    e.err = n->d_err;
    e.g = level_geo(n, l);
    WS_CUDA(n, wsn::conv(d.cout_p, d.cin_p, gout, n->wst + d.wb, n->wst + d.wbt, e, n->stream));
    return LBM_OK;
}

// weight and bias gradients of layer k from its input activation and output gradient
int bwd_weight(lbm_wsnet* n, int k, const bf16* act, const bf16* gout, int l) {
    const wsn::LayerDesc& d = n->L[k];
    wsn::WgArgs a{};
    a.gw = n->g + d.woff;
    a.cin_real = d.cin;
    a.cout_real = d.cout;
    a.err = n->d_err;
    a.g = level_geo(n, l);
    const int64_t rows = a.g.rows();
    const unsigned nb = (unsigned)std::min<int64_t>(std::max<int64_t>(1, rows / 512), 152 * 4);
    // partial sums per row split, added in a fixed order: the gradients (and so
    // the training) do not depend on the order in which CTAs finish
    const int64_t need = std::max<int64_t>(wsn::wgrad_splits(d.cin_p, d.cout_p, rows, n->n_sm) * d.cout * 27 * d.cin,
                                           (int64_t)nb * d.cout);
    if (need > n->part_cap) {
        WS_CUDA(n, cudaStreamSynchronize(n->stream));
        cudaFree(n->part);
        n->part = nullptr;
        n->part_cap = 0;
        if (cudaMalloc(&n->part, sizeof(float) * need) != cudaSuccess)
            return wfail(n, LBM_ENOMEM, "gradient partial sums (%lld floats)", (long long)need);
        n->part_cap = need;
    }
    a.part = n->part;
    a.part_cap = n->part_cap;
    WS_CUDA(n, wsn::wgrad(d.cin_p, d.cout_p, act, gout, a, n->stream, n->n_sm));
    wsn::k_bias_grad<<<nb, 256, 0, n->stream>>>(gout, rows, d.cout_p, d.cout, n->g + d.boff, n->part);
    wsn::k_split_sum<<<wsn::gs_blocks(d.cout), 256, 0, n->stream>>>(n->part, nb, d.cout, n->g + d.boff);
    WS_CUDA(n, cudaGetLastError());
    return LBM_OK;
}

// Forward pass of the batch whose masks are in buffer "M"; keeps activations.
int forward(lbm_wsnet* n) {
    using namespace wsn;
    if (!n->packed) {
        int rc = pack_weights(n);
        if (rc) return rc;
    }
    const int Lv = n->levels;
    cudaStream_t st = n->stream;
    const PGeo g0 = level_geo(n, 0);
    k_x32<<<gs_blocks((int64_t)g0.B * g0.X * g0.Y * g0.Z), 256, 0, st>>>((const uint8_t*)n->buf.at("M"),
                                                                         B16(n, "X"), g0);
    WS_CUDA(n, cudaGetLastError());
    char s1[32], s2[32], s3[32], s4[32];
    int k = 0, rc;
    const bf16* inp = B16(n, "X");
    for (int l = 0; l < Lv; ++l) {
        if (l > 0) {
            snprintf(s1, sizeof s1, "E%db", l - 1);
            snprintf(s2, sizeof s2, "P%d", l);
            const PGeo gc = level_geo(n, l), gf = level_geo(n, l - 1);
            const int C = chans(n, l - 1);
            k_pool<<<gs_blocks((int64_t)gc.B * gc.X * gc.Y * gc.Z * (C / 8)), 256, 0, st>>>(B16(n, s1), B16(n, s2),
                                                                                            gc, gf, C);
            WS_CUDA(n, cudaGetLastError());
            inp = B16(n, s2);
        }
        snprintf(s1, sizeof s1, "E%da", l);
        snprintf(s2, sizeof s2, "E%db", l);
        if ((rc = fwd_layer(n, k, inp, l, true, B16(n, s1), nullptr, nullptr))) return rc;
        if ((rc = fwd_layer(n, k + 1, B16(n, s1), l, true, B16(n, s2), nullptr, nullptr))) return rc;
        k += 2;
    }
    snprintf(s1, sizeof s1, "E%db", Lv - 1);
    std::string below = s1;
    for (int l = Lv - 2; l >= 0; --l) {
        snprintf(s1, sizeof s1, "U%d", l);
        const PGeo gf = level_geo(n, l), gc = level_geo(n, l + 1);
        const int C = chans(n, l + 1);
        k_up<<<gs_blocks((int64_t)gf.B * gf.X * gf.Y * gf.Z * (C / 8)), 256, 0, st>>>(B16(n, below), B16(n, s1), gf,
                                                                                       gc, C);
        WS_CUDA(n, cudaGetLastError());
        snprintf(s2, sizeof s2, "D%da", l);
        snprintf(s3, sizeof s3, "S%d", l);
        snprintf(s4, sizeof s4, "E%db", l);
        // Dla = relu(conv(Ul)), Sl = Dla + Elb fused into the epilogue
        if ((rc = fwd_layer(n, k, B16(n, s1), l, true, B16(n, s2), B16(n, s4), B16(n, s3)))) return rc;
        snprintf(s1, sizeof s1, "D%db", l);
        if ((rc = fwd_layer(n, k + 1, B16(n, s3), l, true, B16(n, s1), nullptr, nullptr))) return rc;
        below = s1;
        k += 2;
    }
    // Y = conv(top) * X (kOut of the 32 padded output channels)
    if ((rc = fwd_layer(n, k, B16(n, below), 0, false, nullptr, nullptr, nullptr, (float*)n->buf.at("Y"),
                        B16(n, "X"))))
        return rc;
    return LBM_OK;
}

// Backward pass from buffer "gZ"; accumulates parameter gradients into n->g.
int backward(lbm_wsnet* n) {
    using namespace wsn;
    const int Lv = n->levels;
    cudaStream_t st = n->stream;
    const int nl = (int)n->L.size();
    char s1[32], s2[32], s3[32], s4[32];
    int rc, k = nl - 1;
    std::string top = Lv > 1 ? "D0b" : "E0b";
    // output layer: weights from (top, gZ); gradient w.r.t. top, masked by relu'(top)
    if ((rc = bwd_weight(n, k, B16(n, top), B16(n, "gZ"), 0))) return rc;
    if ((rc = bwd_data(n, k, B16(n, "gZ"), 0, nullptr, B16(n, top), B16(n, "gA0")))) return rc;
    k -= 1;
    std::string g = "gA0";  // gradient w.r.t. the pre-activation output of the next layer back
    for (int l = 0; l <= Lv - 2; ++l) {
        // Dlb = relu(conv(Sl)):  weight grad from (Sl, g); gS = W^T g -> skip gradient and (gS * relu'(Dla))
        snprintf(s1, sizeof s1, "S%d", l);
        snprintf(s2, sizeof s2, "gskip%d", l);
        snprintf(s3, sizeof s3, "D%da", l);
        snprintf(s4, sizeof s4, "gB%d", l);
        if ((rc = bwd_weight(n, k, B16(n, s1), B16(n, g), l))) return rc;
        if ((rc = bwd_data(n, k, B16(n, g), l, B16(n, s2), B16(n, s3), B16(n, s4)))) return rc;
        // Dla = relu(conv(Ul)): weight grad from (Ul, gB); gU = W^T gB
        snprintf(s1, sizeof s1, "U%d", l);
        snprintf(s3, sizeof s3, "gU%d", l);
        if ((rc = bwd_weight(n, k - 1, B16(n, s1), B16(n, s4), l))) return rc;
        if ((rc = bwd_data(n, k - 1, B16(n, s4), l, B16(n, s3), nullptr, nullptr))) return rc;
        // into level l+1: (adjoint of up) * relu'(D(l+1)b or E(L-1)b)
        const PGeo gc = level_geo(n, l + 1), gf = level_geo(n, l);
        const int C = chans(n, l + 1);
        if (l + 1 == Lv - 1) snprintf(s1, sizeof s1, "E%db", l + 1);
        else snprintf(s1, sizeof s1, "D%db", l + 1);
        snprintf(s2, sizeof s2, "gA%d", l + 1);
        k_up_bwd_mask<<<gs_blocks((int64_t)gc.B * gc.X * gc.Y * gc.Z * (C / 8)), 256, 0, st>>>(
            B16(n, s3), B16(n, s1), B16(n, s2), gc, gf, C);
        WS_CUDA(n, cudaGetLastError());
        g = s2;
        k -= 2;
    }
    for (int l = Lv - 1; l >= 0; --l) {
        // Elb = relu(conv(Ela)); g is the gradient w.r.t. its pre-activation output
        snprintf(s1, sizeof s1, "E%da", l);
        snprintf(s2, sizeof s2, "gB%d", l);
        if ((rc = bwd_weight(n, k, B16(n, s1), B16(n, g), l))) return rc;
        if ((rc = bwd_data(n, k, B16(n, g), l, nullptr, B16(n, s1), B16(n, s2)))) return rc;
        // Ela = relu(conv(Pl or X))
        std::string inp = "X";
        if (l > 0) {
            snprintf(s3, sizeof s3, "P%d", l);
            inp = s3;
        }
        if ((rc = bwd_weight(n, k - 1, B16(n, inp), B16(n, s2), l))) return rc;
        if (l > 0) {
            snprintf(s4, sizeof s4, "gP%d", l);
            if ((rc = bwd_data(n, k - 1, B16(n, s2), l, B16(n, s4), nullptr, nullptr))) return rc;
            // into level l-1: (skip gradient + adjoint of pool) * relu'(E(l-1)b)
            const PGeo gf = level_geo(n, l - 1), gc = level_geo(n, l);
            const int C = chans(n, l - 1);
            snprintf(s1, sizeof s1, "gskip%d", l - 1);
            snprintf(s2, sizeof s2, "E%db", l - 1);
            snprintf(s3, sizeof s3, "gA%d", l - 1);
            k_pool_bwd_add_mask<<<gs_blocks((int64_t)gf.B * gf.X * gf.Y * gf.Z * (C / 8)), 256, 0, st>>>(
                B16(n, s4), B16(n, s1), B16(n, s2), B16(n, s3), gf, gc, C);
            WS_CUDA(n, cudaGetLastError());
            g = s3;
        }
        k -= 2;
    }
    return LBM_OK;
}

int check_err(lbm_wsnet* n) {
    int h = 0;
    WS_CUDA(n, cudaMemcpyAsync(&h, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    WS_CUDA(n, cudaStreamSynchronize(n->stream));
    if (h) {
        cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream);
        return wfail(n, LBM_ETIMEOUT, "a tensor-core pipeline wait ran out (bounded at ~1 s)");
    }
    return LBM_OK;
}

bool dims_ok(const lbm_wsnet* n, int nz, int ny, int nx) {
    const int q = 1 << (n->levels - 1);
    return nz >= q && ny >= q && nx >= q && nz % q == 0 && ny % q == 0 && nx % q == 0;
}

// loss and gradient of the batch already in buffers "M" (masks) and "T" (targets)
int loss_grad_dev(lbm_wsnet* n, int64_t npore, double* loss) {
    if (npore <= 0) return wfail(n, LBM_EINVAL, "no pore voxels");
    int rc = forward(n);
    if (rc) return rc;
    const PGeo g0 = level_geo(n, 0);
    WS_CUDA(n, cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream));
    wsn::k_mse<<<wsn::gs_blocks((int64_t)g0.B * g0.X * g0.Y * g0.Z), 256, 0, n->stream>>>(
        (const float*)n->buf.at("Y"), (const float*)n->buf.at("T"), B16(n, "X"), B16(n, "gZ"), g0,
        1.0 / ((double)wsn::kOut * (double)npore), n->d_loss);
    WS_CUDA(n, cudaGetLastError());
    WS_CUDA(n, cudaMemsetAsync(n->g, 0, sizeof(float) * n->np, n->stream));
    if ((rc = backward(n))) return rc;
    if (loss) WS_CUDA(n, cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    return LBM_OK;
}

int64_t count_pores(const uint8_t* masks, int64_t n) {
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) c += masks[i] == 0;
    return c;
}

}  // namespace

extern "C" {

int lbm_wsnet_create(int levels, int base, lbm_wsnet** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (levels < 1 || levels > 4 || !wsn::chan_ok(base) || !wsn::chan_ok(base << (levels - 1))) return LBM_EINVAL;
    auto* n = new (std::nothrow) lbm_wsnet();
    if (!n) return LBM_ENOMEM;
    cudaGetDevice(&n->device);
    cudaDeviceGetAttribute(&n->n_sm, cudaDevAttrMultiProcessorCount, n->device);
    n->levels = levels;
    n->base = base;
    std::vector<std::pair<int, int>> shp;  // (cout, cin) in forward order
    shp.push_back({base, 1});
    shp.push_back({base, base});
    for (int l = 1; l < levels; ++l) {
        shp.push_back({base << l, base << (l - 1)});
        shp.push_back({base << l, base << l});
    }
    for (int l = levels - 2; l >= 0; --l) {
        shp.push_back({base << l, base << (l + 1)});
        shp.push_back({base << l, base << l});
    }
    shp.push_back({wsn::kOut, base});
    int64_t k = 0, w = 0, b = 0;
    for (auto& s : shp) {
        wsn::LayerDesc d{};
        d.cout = s.first;
        d.cin = s.second;
        d.cout_p = std::max(32, d.cout);
        d.cin_p = std::max(32, d.cin);
        d.woff = k;
        k += (int64_t)d.cout * 27 * d.cin;
        d.boff = k;
        k += d.cout;
        d.wf = w;
        w += (int64_t)d.cout_p * 27 * d.cin_p;
        d.wb = w;
        w += (int64_t)d.cout_p * 27 * d.cin_p;
        d.wft = w;
        w += (int64_t)d.cout_p * 27 * d.cin_p;
        d.wbt = w;
        w += (int64_t)d.cout_p * 27 * d.cin_p;
        d.bp = b;
        b += d.cout_p;
        n->L.push_back(d);
    }
    n->np = k;
    n->nw = w;
    n->nb = b;
    cudaError_t e = cudaMalloc(&n->p, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->g, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->wst, w * 2);
    if (e == cudaSuccess) e = cudaMalloc(&n->bst, b * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->d_L, sizeof(wsn::LayerDesc) * n->L.size());
    if (e == cudaSuccess) e = cudaMalloc(&n->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&n->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(n->p, 0, k * 4);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, k * 4);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, k * 4);
    if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(n->d_L, n->L.data(), sizeof(wsn::LayerDesc) * n->L.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lbm_wsnet_destroy(n);
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
    *out = n;
    return LBM_OK;
}

int lbm_wsnet_num_params(const lbm_wsnet* n, int64_t* np) {
    if (!n || !np) return LBM_EINVAL;
    *np = n->np;
    return LBM_OK;
}

int lbm_wsnet_set_stream(lbm_wsnet* n, void* s) {
    int rc = wenter(n);
    if (rc) return rc;
    n->stream = (cudaStream_t)s;
    return LBM_OK;
}

int lbm_wsnet_set_params(lbm_wsnet* n, const float* host) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!host) return wfail(n, LBM_EINVAL, "NULL params");
    WS_CUDA(n, cudaStreamSynchronize(n->stream));
    WS_CUDA(n, cudaMemcpy(n->p, host, n->np * 4, cudaMemcpyHostToDevice));
    WS_CUDA(n, cudaMemset(n->m, 0, n->np * 4));
    WS_CUDA(n, cudaMemset(n->v, 0, n->np * 4));
    n->adam_t = 0;
    n->packed = false;
    return LBM_OK;
}

int lbm_wsnet_get_params(lbm_wsnet* n, float* host) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!host) return wfail(n, LBM_EINVAL, "NULL params");
    WS_CUDA(n, cudaStreamSynchronize(n->stream));
    WS_CUDA(n, cudaMemcpy(host, n->p, n->np * 4, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int lbm_wsnet_loss_grad(lbm_wsnet* n, const uint8_t* mask, const float* target, int batch, int nx, int ny, int nz,
                        double* loss, float* grad) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!mask || !target || batch < 1 || !dims_ok(n, nz, ny, nx))
        return wfail(n, LBM_EINVAL, "bad arguments (sides must be multiples of %d)", 1 << (n->levels - 1));
    const int64_t N0 = (int64_t)nz * ny * nx;
    if ((rc = ensure_buffers(n, batch, nx, ny, nz, true))) return rc;
    WS_CUDA(n, cudaMemcpyAsync(n->buf.at("M"), mask, batch * N0, cudaMemcpyHostToDevice, n->stream));
    WS_CUDA(n, cudaMemcpyAsync(n->buf.at("T"), target, batch * wsn::kOut * N0 * 4, cudaMemcpyHostToDevice,
                               n->stream));
    double l = 0.0;
    if ((rc = loss_grad_dev(n, count_pores(mask, batch * N0), &l))) return rc;
    if ((rc = check_err(n))) return rc;
    if (loss) *loss = l;
    if (grad) WS_CUDA(n, cudaMemcpy(grad, n->g, n->np * 4, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int lbm_wsnet_train(lbm_wsnet* n, const uint8_t* masks, const float* targets, int n_samples, int nx, int ny, int nz,
                    int epochs, int batch, float lr, const int* order, float* loss_history) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!masks || !targets || n_samples < 1 || epochs < 1 || batch < 1 || !dims_ok(n, nz, ny, nx) || !order)
        return wfail(n, LBM_EINVAL, "bad arguments");
    const int64_t N0 = (int64_t)nz * ny * nx;
    for (int64_t i = 0; i < (int64_t)epochs * n_samples; ++i)
        if (order[i] < 0 || order[i] >= n_samples) return wfail(n, LBM_EINVAL, "order[%lld] out of range", (long long)i);
    std::vector<int64_t> npore(n_samples);
    for (int s = 0; s < n_samples; ++s) npore[s] = count_pores(masks + s * N0, N0);
    uint8_t* dm = nullptr;
    float* dt = nullptr;
    WS_CUDA(n, cudaMalloc(&dm, (size_t)n_samples * N0));
    cudaError_t e = cudaMalloc(&dt, (size_t)n_samples * wsn::kOut * N0 * 4);
    if (e != cudaSuccess) {
        cudaFree(dm);
        return wfail(n, LBM_ENOMEM, "training set: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(dm, masks, (size_t)n_samples * N0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dt, targets, (size_t)n_samples * wsn::kOut * N0 * 4, cudaMemcpyHostToDevice);
    double* h_loss = nullptr;
    const int nbatch = (n_samples + batch - 1) / batch;
    if (e == cudaSuccess) e = cudaMallocHost(&h_loss, sizeof(double) * (size_t)epochs * nbatch);
    for (int ep = 0; ep < epochs && rc == LBM_OK && e == cudaSuccess; ++ep) {
        for (int bi = 0; bi < nbatch && rc == LBM_OK; ++bi) {
            const int s0 = bi * batch;
            const int B = std::min(batch, n_samples - s0);
            if ((rc = ensure_buffers(n, B, nx, ny, nz, true))) break;
            int64_t np_b = 0;
            for (int j = 0; j < B && e == cudaSuccess; ++j) {
                const int idx = order[(size_t)ep * n_samples + s0 + j];
                np_b += npore[idx];
                e = cudaMemcpyAsync((uint8_t*)n->buf.at("M") + (size_t)j * N0, dm + (size_t)idx * N0, N0,
                                    cudaMemcpyDeviceToDevice, n->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync((float*)n->buf.at("T") + (size_t)j * wsn::kOut * N0,
                                        dt + (size_t)idx * wsn::kOut * N0, wsn::kOut * N0 * 4,
                                        cudaMemcpyDeviceToDevice, n->stream);
            }
            if (e != cudaSuccess) break;
            if ((rc = loss_grad_dev(n, np_b, h_loss + (size_t)ep * nbatch + bi))) break;
            ++n->adam_t;
            const float b1 = 0.9f, b2 = 0.999f;
            wsn::k_adam<<<wsn::gs_blocks(n->np), 256, 0, n->stream>>>(
                n->p, n->g, n->m, n->v, n->np, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)n->adam_t),
                1.f - powf(b2, (float)n->adam_t));
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((rc = pack_weights(n))) break;
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(n->stream);
    if (e == cudaSuccess) e = e2;
    if (rc == LBM_OK && e == cudaSuccess) rc = check_err(n);
    if (rc == LBM_OK && e == cudaSuccess && loss_history)
        for (int ep = 0; ep < epochs; ++ep) {
            double s = 0.0;
            for (int bi = 0; bi < nbatch; ++bi) s += h_loss[(size_t)ep * nbatch + bi];
            loss_history[ep] = (float)(s / nbatch);
        }
    cudaFree(dm);
    cudaFree(dt);
    if (h_loss) cudaFreeHost(h_loss);
    if (rc) return rc;
    if (e != cudaSuccess) return wfail(n, LBM_ECUDA, "lbm_wsnet_train: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_wsnet_predict(lbm_wsnet* n, const uint8_t* mask, int nx, int ny, int nz, float* y) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!mask || !y || !dims_ok(n, nz, ny, nx))
        return wfail(n, LBM_EINVAL, "bad arguments (sides multiple of %d)", 1 << (n->levels - 1));
    const int64_t N0 = (int64_t)nz * ny * nx;
    if ((rc = ensure_buffers(n, 1, nx, ny, nz, false))) return rc;
    WS_CUDA(n, cudaMemcpyAsync(n->buf.at("M"), mask, N0, cudaMemcpyHostToDevice, n->stream));
    if ((rc = forward(n))) return rc;
    WS_CUDA(n, cudaMemcpyAsync(y, n->buf.at("Y"), wsn::kOut * N0 * 4, cudaMemcpyDeviceToHost, n->stream));
    return check_err(n);
}

int lbm_wsnet_release_buffers(lbm_wsnet* n) {
    int rc = wenter(n);
    if (rc) return rc;
    cudaStreamSynchronize(n->stream);
    free_buffers(n);
    cudaFree(n->part);
    n->part = nullptr;
    n->part_cap = 0;
    return LBM_OK;
}

int lbm_wsnet_destroy(lbm_wsnet* n) {
    if (!n) return LBM_OK;
    cudaSetDevice(n->device);
    if (n->stream) cudaStreamSynchronize(n->stream);
    free_buffers(n);
    cudaFree(n->p);
    cudaFree(n->g);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->wst);
    cudaFree(n->bst);
    cudaFree(n->d_L);
    cudaFree(n->d_loss);
    cudaFree(n->part);
    cudaFree(n->d_err);
    delete n;
    return LBM_OK;
}

const char* lbm_wsnet_last_error(const lbm_wsnet* n) { return n ? n->err.c_str() : "invalid network handle"; }

}  // extern "C"

namespace {

// One convolution on caller buffers, launched `reps` times; with ms != NULL the
// launches are bracketed by CUDA events on `st` and the mean time returned.
int conv_call(int op, const void* in, const void* aux, const void* w, const float* bias, int relu, void* out,
              int batch, int nx, int ny, int nz, int cin, int cout, int reps, float* ms, cudaStream_t st) {
    if (!in || !w || !out || batch < 1 || nx < 1 || ny < 1 || nz < 1 || !wsn::chan_ok(cin) || !wsn::chan_ok(cout) ||
        op < 0 || op > 2 || (op == 2 && !aux) || reps < 1)
        return LBM_EINVAL;
    const PGeo g{batch, nx, ny, nz};
    int* d_err = nullptr;
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return LBM_ENOMEM;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    // the layouts the convolution kernel reads: forward [cout][27][cin] and
    // [27][cout][cin]; data gradient (flipped taps) [cin][27][cout] and [27][cin][cout]
    bf16* wb = nullptr;  // two arrays: wb and wb + n
    const size_t nw = (size_t)cout * 27 * cin;
    if (e == cudaSuccess && op < 2) {
        std::vector<uint16_t> hw(nw), hb(2 * nw);
        e = cudaMemcpyAsync(hw.data(), w, nw * 2, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int co = 0; co < cout && e == cudaSuccess; ++co)
            for (int t = 0; t < 27; ++t)
                for (int ci = 0; ci < cin; ++ci) {
                    const uint16_t v = hw[((size_t)co * 27 + t) * cin + ci];
                    if (op == 0) {
                        hb[((size_t)co * 27 + t) * cin + ci] = v;
                        hb[nw + ((size_t)t * cout + co) * cin + ci] = v;
                    } else {
                        hb[((size_t)ci * 27 + (26 - t)) * cout + co] = v;
                        hb[nw + ((size_t)(26 - t) * cin + ci) * cout + co] = v;
                    }
                }
        if (e == cudaSuccess) e = cudaMalloc(&wb, hb.size() * 2);
        if (e == cudaSuccess) e = cudaMemcpyAsync(wb, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, st);
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ms && e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (ms && e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (ms && e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        if (op == 0) {
            wsn::ConvEpi ep{};
            ep.bias = bias;
            ep.relu = relu;
            ep.out = (bf16*)out;
            ep.err = d_err;
            ep.g = g;
            e = wsn::conv(cin, cout, (const bf16*)in, wb, wb + nw, ep, st);
        } else if (op == 1) {
            wsn::ConvEpi ep{};
            ep.out = (bf16*)out;
            ep.err = d_err;
            ep.g = g;
            e = wsn::conv(cout, cin, (const bf16*)in, wb, wb + nw, ep, st);
        } else {
            wsn::WgArgs a{};
            a.gw = (float*)out;
            a.cin_real = cin;
            a.cout_real = cout;
            a.err = d_err;
            a.g = g;
            e = wsn::wgrad(cin, cout, (const bf16*)in, (const bf16*)aux, a, st, nsm);
        }
    }
    if (ms && e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ms && e == cudaSuccess) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        *ms = t / reps;
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(d_err);
    if (wb) cudaFree(wb);
    if (e != cudaSuccess) return LBM_ECUDA;
    return h ? LBM_ETIMEOUT : LBM_OK;
}

}  // namespace

extern "C" {

int lbm_conv3d_bf16(int op, const void* in, const void* aux, const void* w, const float* bias, int relu, void* out,
                    int batch, int nx, int ny, int nz, int cin, int cout, void* stream) {
    return conv_call(op, in, aux, w, bias, relu, out, batch, nx, ny, nz, cin, cout, 1, nullptr,
                     (cudaStream_t)stream);
}

int lbm_conv3d_bf16_time(int op, const void* in, const void* aux, const void* w, const float* bias, int relu,
                         void* out, int batch, int nx, int ny, int nz, int cin, int cout, int reps, float* ms,
                         void* stream) {
    if (!ms) return LBM_EINVAL;
    return conv_call(op, in, aux, w, bias, relu, out, batch, nx, ny, nz, cin, cout, reps, ms,
                     (cudaStream_t)stream);
}

}  // extern "C"
