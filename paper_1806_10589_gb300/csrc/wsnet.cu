// Learned warm start: a small 3-D U-Net that predicts the steady velocity field
// u / u_D of a pore geometry, trained on steady states this library computes,
// with its own CUDA forward, backward and Adam kernels (FP32, CUDA cores).
//
// Architecture (channels c0, c1, c2; every box side divisible by 4):
//   L0a = relu(conv(X)), L0b = relu(conv(L0a))              full resolution
//   L1a = relu(conv(pool(L0b))), L1b = relu(conv(L1a))       1/2
//   L2a = relu(conv(pool(L1b))), L2b = relu(conv(L2a))       1/4
//   L3a = relu(conv(up(L2b))),   L3b = relu(conv(L3a + L1b)) 1/2
//   L4a = relu(conv(up(L3b))),   L4b = relu(conv(L4a + L0b)) full
//   Y   = conv(L4b) * X          (3 channels; X = pore indicator)
// conv = 3x3x3 cross-correlation, zero padding, bias; pool = 2x2x2 mean;
// up = nearest 2x.  Loss = masked mean squared error over pore voxels.
// Tensors are [B][C][nz][ny][nx] float32.  Parameters: per layer W[co][ci][27]
// (taps dz, dy, dx in -1..1) then b[co].
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace wsn {
namespace {

constexpr int TZ = 4, TY = 8, TX = 8;      // output tile of the conv kernels
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;
constexpr int kThreads = TZ * TY * TX;     // 256
constexpr int kLayers = 11;

struct Geo {
    int nz, ny, nx;
    int tz, ty, tx;  // tile counts
    __host__ __device__ int64_t vox() const { return (int64_t)nz * ny * nx; }
    __host__ __device__ int tiles() const { return tz * ty * tx; }
};
Geo make_geo(int nz, int ny, int nx) {
    return Geo{nz, ny, nx, (nz + TZ - 1) / TZ, (ny + TY - 1) / TY, (nx + TX - 1) / TX};
}

// Load the (TZ+2)x(TY+2)x(TX+2) halo of channel plane `src` around tile t.
__device__ __forceinline__ void load_halo(float (*tile)[HY][HX], const float* __restrict__ src, const Geo& g,
                                          int z0, int y0, int x0) {
    for (int k = threadIdx.x; k < HZ * HY * HX; k += kThreads) {
        const int hx = k % HX, hy = (k / HX) % HY, hz = k / (HX * HY);
        const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
        float v = 0.f;
        if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz)
            v = src[((int64_t)gz * g.ny + gy) * g.nx + gx];
        tile[hz][hy][hx] = v;
    }
}

// out[b][co] = act(bias[co] + sum_ci sum_t W[co][ci][t] in[b][ci](x + t)); grid (tiles, B).
template <int COUT>
__global__ void __launch_bounds__(kThreads)
k_conv_fwd(const float* __restrict__ in, int cin, const float* __restrict__ W, const float* __restrict__ bias,
           float* __restrict__ out, Geo g, int relu) {
    __shared__ float tile[HZ][HY][HX];
    __shared__ float ws[COUT * 27];
    int t = blockIdx.x;
    const int tx = t % g.tx;
    t /= g.tx;
    const int ty = t % g.ty, tz = t / g.ty;
    const int b = blockIdx.y;
    const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
    const int x = tx * TX + lx, y = ty * TY + ly, z = tz * TZ + lz;
    const bool on = x < g.nx && y < g.ny && z < g.nz;
    const int64_t N = g.vox();
    float acc[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc[c] = 0.f;
    for (int ci = 0; ci < cin; ++ci) {
        load_halo(tile, in + ((int64_t)b * cin + ci) * N, g, tz * TZ, ty * TY, tx * TX);
        for (int k = threadIdx.x; k < COUT * 27; k += kThreads) ws[k] = W[((k / 27) * cin + ci) * 27 + k % 27];
        __syncthreads();
        if (on) {
            float v[27];
#pragma unroll
            for (int q = 0; q < 27; ++q) v[q] = tile[lz + q / 9][ly + (q / 3) % 3][lx + q % 3];
#pragma unroll
            for (int c = 0; c < COUT; ++c) {
                float s = acc[c];
#pragma unroll
                for (int q = 0; q < 27; ++q) s = fmaf(ws[c * 27 + q], v[q], s);
                acc[c] = s;
            }
        }
        __syncthreads();
    }
    if (on) {
        const int64_t o = ((int64_t)z * g.ny + y) * g.nx + x;
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
            float r = acc[c] + (bias ? bias[c] : 0.f);
            if (relu) r = fmaxf(r, 0.f);
            out[((int64_t)b * COUT + c) * N + o] = r;
        }
    }
}

// gW[co][ci][t] += sum_x g[b][co](x) in[b][ci](x + t) over one tile; grid (tiles, B*cin).
template <int COUT>
__global__ void __launch_bounds__(kThreads)
k_conv_bwd_w(const float* __restrict__ in, int cin, const float* __restrict__ gout, float* __restrict__ gW, Geo g) {
    __shared__ float tile[HZ][HY][HX];
    __shared__ float gs[COUT][kThreads];
    int t = blockIdx.x;
    const int tx = t % g.tx;
    t /= g.tx;
    const int ty = t % g.ty, tz = t / g.ty;
    const int ci = blockIdx.y % cin, b = blockIdx.y / cin;
    const int64_t N = g.vox();
    load_halo(tile, in + ((int64_t)b * cin + ci) * N, g, tz * TZ, ty * TY, tx * TX);
    {
        const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
        const int x = tx * TX + lx, y = ty * TY + ly, z = tz * TZ + lz;
        const bool on = x < g.nx && y < g.ny && z < g.nz;
        const int64_t o = ((int64_t)z * g.ny + y) * g.nx + x;
        for (int c = 0; c < COUT; ++c) gs[c][threadIdx.x] = on ? gout[((int64_t)b * COUT + c) * N + o] : 0.f;
    }
    __syncthreads();
    for (int pr = threadIdx.x; pr < COUT * 27; pr += kThreads) {
        const int c = pr / 27, q = pr % 27;
        const int dz = q / 9, dy = (q / 3) % 3, dx = q % 3;
        float s = 0.f;
        for (int v = 0; v < kThreads; ++v) {
            const int lx = v % TX, ly = (v / TX) % TY, lz = v / (TX * TY);
            s = fmaf(gs[c][v], tile[lz + dz][ly + dy][lx + dx], s);
        }
        atomicAdd(gW + ((int64_t)c * cin + ci) * 27 + q, s);
    }
}

// gb[c] += sum over a chunk of voxels of g[b][c]; grid (chunks, B*C).
__global__ void k_bias_grad(const float* __restrict__ gout, int C, int64_t N, float* __restrict__ gb) {
    __shared__ float sh[32];
    const int c = blockIdx.y % C, b = blockIdx.y / C;
    const float* src = gout + ((int64_t)b * C + c) * N;
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        s += src[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(gb + c, s);
    }
}

// Wt[ci][co][26 - t] = W[co][ci][t]: the backward-data convolution's weights.
__global__ void k_flip_weights(const float* __restrict__ W, int cout, int cin, float* __restrict__ Wt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cout * cin * 27) return;
    const int t = k % 27, ci = (k / 27) % cin, co = k / (27 * cin);
    Wt[((int64_t)ci * cout + co) * 27 + (26 - t)] = W[k];
}

__global__ void k_pool(const float* __restrict__ in, float* __restrict__ out, int64_t BC, Geo go) {
    const int64_t n = BC * go.vox();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % go.nx), y = (int)((k / go.nx) % go.ny), z = (int)((k / ((int64_t)go.nx * go.ny)) % go.nz);
        const int64_t bc = k / go.vox();
        const int nx = 2 * go.nx, ny = 2 * go.ny;
        const float* s = in + bc * (int64_t)8 * go.vox();
        float a = 0.f;
        for (int d = 0; d < 8; ++d)
            a += s[((int64_t)(2 * z + (d >> 2)) * ny + (2 * y + ((d >> 1) & 1))) * nx + 2 * x + (d & 1)];
        out[k] = a * 0.125f;
    }
}
__global__ void k_pool_bwd(const float* __restrict__ g, float* __restrict__ gin, int64_t BC, Geo gi) {
    const int64_t n = BC * gi.vox();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % gi.nx), y = (int)((k / gi.nx) % gi.ny), z = (int)((k / ((int64_t)gi.nx * gi.ny)) % gi.nz);
        const int64_t bc = k / gi.vox();
        const int64_t co = bc * (gi.vox() / 8) + ((int64_t)(z / 2) * (gi.ny / 2) + y / 2) * (gi.nx / 2) + x / 2;
        gin[k] += 0.125f * g[co];
    }
}
__global__ void k_up(const float* __restrict__ in, float* __restrict__ out, int64_t BC, Geo go) {
    const int64_t n = BC * go.vox();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % go.nx), y = (int)((k / go.nx) % go.ny), z = (int)((k / ((int64_t)go.nx * go.ny)) % go.nz);
        const int64_t bc = k / go.vox();
        out[k] = in[bc * (go.vox() / 8) + ((int64_t)(z / 2) * (go.ny / 2) + y / 2) * (go.nx / 2) + x / 2];
    }
}
__global__ void k_up_bwd(const float* __restrict__ g, float* __restrict__ gin, int64_t BC, Geo gi) {
    const int64_t n = BC * gi.vox();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % gi.nx), y = (int)((k / gi.nx) % gi.ny), z = (int)((k / ((int64_t)gi.nx * gi.ny)) % gi.nz);
        const int64_t bc = k / gi.vox();
        const int nx = 2 * gi.nx, ny = 2 * gi.ny;
        const float* s = g + bc * (int64_t)8 * gi.vox();
        float a = 0.f;
        for (int d = 0; d < 8; ++d)
            a += s[((int64_t)(2 * z + (d >> 2)) * ny + (2 * y + ((d >> 1) & 1))) * nx + 2 * x + (d & 1)];
        gin[k] = a;
    }
}
__global__ void k_add(const float* a, const float* b, float* out, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = a[k] + b[k];
}
// g *= (act > 0)
__global__ void k_relu_mask(float* g, const float* act, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (!(act[k] > 0.f)) g[k] = 0.f;
}
// y[b][c] *= X[b]
__global__ void k_mask_mul(float* y, const float* X, int C, int64_t N, int64_t B) {
    const int64_t n = B * C * N;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] *= X[(k / (C * N)) * N + k % N];
}
// X[b][x] = 1 - mask[b][x]
__global__ void k_pore_from_mask(const uint8_t* m, float* X, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        X[k] = m[k] ? 0.f : 1.f;
}
// masked MSE: gY = 2 (Y - T) X / (3 npore), loss += sum (Y - T)^2 X / (3 npore)
__global__ void k_mse(const float* Y, const float* T, const float* X, int64_t N, int64_t B, double inv,
                      float* gY, double* loss) {
    __shared__ double sh[32];
    const int64_t n = B * 3 * N;
    double s = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float xm = X[(k / (3 * N)) * N + k % N];
        const float d = (Y[k] - T[k]) * xm;
        gY[k] = (float)(2.0 * inv) * d;
        s += (double)d * d;
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
__global__ void k_count(const float* X, int64_t n, unsigned long long* cnt) {
    unsigned long long c = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        c += X[k] > 0.5f;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(cnt, c);
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

inline unsigned gs_blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32); }

template <int C>
cudaError_t conv_fwd_t(const float* in, int cin, const float* W, const float* b, float* out, const Geo& g, int B,
                       int relu, cudaStream_t st) {
    k_conv_fwd<C><<<dim3((unsigned)g.tiles(), (unsigned)B), kThreads, 0, st>>>(in, cin, W, b, out, g, relu);
    return cudaGetLastError();
}
cudaError_t conv_fwd(int cout, const float* in, int cin, const float* W, const float* b, float* out, const Geo& g,
                     int B, int relu, cudaStream_t st) {
    switch (cout) {
        case 3: return conv_fwd_t<3>(in, cin, W, b, out, g, B, relu, st);
        case 8: return conv_fwd_t<8>(in, cin, W, b, out, g, B, relu, st);
        case 16: return conv_fwd_t<16>(in, cin, W, b, out, g, B, relu, st);
        case 32: return conv_fwd_t<32>(in, cin, W, b, out, g, B, relu, st);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t conv_bwd_w(int cout, const float* in, int cin, const float* gout, float* gW, const Geo& g, int B,
                       cudaStream_t st) {
    const dim3 grid((unsigned)g.tiles(), (unsigned)(B * cin));
    switch (cout) {
        case 3: k_conv_bwd_w<3><<<grid, kThreads, 0, st>>>(in, cin, gout, gW, g); break;
        case 8: k_conv_bwd_w<8><<<grid, kThreads, 0, st>>>(in, cin, gout, gW, g); break;
        case 16: k_conv_bwd_w<16><<<grid, kThreads, 0, st>>>(in, cin, gout, gW, g); break;
        case 32: k_conv_bwd_w<32><<<grid, kThreads, 0, st>>>(in, cin, gout, gW, g); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace wsn

struct lbm_wsnet {
    int device = 0;
    int c[3] = {8, 16, 32};
    int co[wsn::kLayers], ci[wsn::kLayers];
    int64_t woff[wsn::kLayers], boff[wsn::kLayers];
    int64_t np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *wt = nullptr;
    double* d_loss = nullptr;
    unsigned long long* d_cnt = nullptr;
    int64_t adam_t = 0;
    cudaStream_t stream = nullptr;
    // activation / gradient buffers keyed by name, sized for (B, geometry)
    std::map<std::string, float*> buf;
    std::map<std::string, size_t> cap;
    std::string err;
    int status = LBM_OK;
};

namespace {

int wfail(lbm_wsnet* n, int code, const char* fmt, ...) {
    static thread_local std::string create_err;
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
#define WS_CUDA(n, call)                                                                      \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return wfail((n), LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int wenter(lbm_wsnet* n) {
    if (!n) return LBM_EINVAL;
    if (n->status == LBM_ECUDA) return LBM_ECUDA;
    WS_CUDA(n, cudaSetDevice(n->device));
    return LBM_OK;
}

float* buffer(lbm_wsnet* n, const std::string& name, size_t floats, cudaError_t* e) {
    auto it = n->buf.find(name);
    if (it != n->buf.end() && n->cap[name] >= floats) return it->second;
    if (it != n->buf.end()) {
        cudaFree(it->second);
        n->buf.erase(it);
    }
    float* d = nullptr;
    *e = cudaMalloc(&d, std::max<size_t>(floats, 1) * sizeof(float));
    if (*e != cudaSuccess) return nullptr;
    n->buf[name] = d;
    n->cap[name] = floats;
    return d;
}

// Forward pass for B samples on geometry (nz, ny, nx); keeps activations.
int forward(lbm_wsnet* n, const uint8_t* d_mask, int B, int nz, int ny, int nx) {
    using namespace wsn;
    const Geo g0 = make_geo(nz, ny, nx), g1 = make_geo(nz / 2, ny / 2, nx / 2), g2 = make_geo(nz / 4, ny / 4, nx / 4);
    const int64_t N0 = g0.vox(), N1 = g1.vox(), N2 = g2.vox();
    const int c0 = n->c[0], c1 = n->c[1], c2 = n->c[2];
    cudaError_t e = cudaSuccess;
    auto B_ = [&](const char* name, int64_t fl) { return buffer(n, name, (size_t)(fl * B), &e); };
    float* X = B_("X", N0);
    float* L0a = B_("L0a", c0 * N0);
    float* L0b = B_("L0b", c0 * N0);
    float* P1 = B_("P1", c0 * N1);
    float* L1a = B_("L1a", c1 * N1);
    float* L1b = B_("L1b", c1 * N1);
    float* P2 = B_("P2", c1 * N2);
    float* L2a = B_("L2a", c2 * N2);
    float* L2b = B_("L2b", c2 * N2);
    float* U1 = B_("U1", c2 * N1);
    float* L3a = B_("L3a", c1 * N1);
    float* S1 = B_("S1", c1 * N1);
    float* L3b = B_("L3b", c1 * N1);
    float* U0 = B_("U0", c1 * N0);
    float* L4a = B_("L4a", c0 * N0);
    float* S0 = B_("S0", c0 * N0);
    float* L4b = B_("L4b", c0 * N0);
    float* Y = B_("Y", 3 * N0);
    if (e != cudaSuccess) return wfail(n, LBM_ENOMEM, "network buffers: %s", cudaGetErrorString(e));
    cudaStream_t st = n->stream;
    auto W = [&](int k) { return n->p + n->woff[k]; };
    auto Bi = [&](int k) { return n->p + n->boff[k]; };
    k_pore_from_mask<<<gs_blocks(B * N0), 256, 0, st>>>(d_mask, X, B * N0);
    WS_CUDA(n, conv_fwd(c0, X, 1, W(0), Bi(0), L0a, g0, B, 1, st));
    WS_CUDA(n, conv_fwd(c0, L0a, c0, W(1), Bi(1), L0b, g0, B, 1, st));
    k_pool<<<gs_blocks(B * c0 * N1), 256, 0, st>>>(L0b, P1, (int64_t)B * c0, g1);
    WS_CUDA(n, conv_fwd(c1, P1, c0, W(2), Bi(2), L1a, g1, B, 1, st));
    WS_CUDA(n, conv_fwd(c1, L1a, c1, W(3), Bi(3), L1b, g1, B, 1, st));
    k_pool<<<gs_blocks(B * c1 * N2), 256, 0, st>>>(L1b, P2, (int64_t)B * c1, g2);
    WS_CUDA(n, conv_fwd(c2, P2, c1, W(4), Bi(4), L2a, g2, B, 1, st));
    WS_CUDA(n, conv_fwd(c2, L2a, c2, W(5), Bi(5), L2b, g2, B, 1, st));
    k_up<<<gs_blocks(B * c2 * N1), 256, 0, st>>>(L2b, U1, (int64_t)B * c2, g1);
    WS_CUDA(n, conv_fwd(c1, U1, c2, W(6), Bi(6), L3a, g1, B, 1, st));
    k_add<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(L3a, L1b, S1, (int64_t)B * c1 * N1);
    WS_CUDA(n, conv_fwd(c1, S1, c1, W(7), Bi(7), L3b, g1, B, 1, st));
    k_up<<<gs_blocks(B * c1 * N0), 256, 0, st>>>(L3b, U0, (int64_t)B * c1, g0);
    WS_CUDA(n, conv_fwd(c0, U0, c1, W(8), Bi(8), L4a, g0, B, 1, st));
    k_add<<<gs_blocks(B * c0 * N0), 256, 0, st>>>(L4a, L0b, S0, (int64_t)B * c0 * N0);
    WS_CUDA(n, conv_fwd(c0, S0, c0, W(9), Bi(9), L4b, g0, B, 1, st));
    WS_CUDA(n, conv_fwd(3, L4b, c0, W(10), Bi(10), Y, g0, B, 0, st));
    k_mask_mul<<<gs_blocks(B * 3 * N0), 256, 0, st>>>(Y, X, 3, N0, B);
    WS_CUDA(n, cudaGetLastError());
    return LBM_OK;
}

// Backward pass from gY (in buffer "gY"); accumulates parameter gradients into n->g.
int backward(lbm_wsnet* n, int B, int nz, int ny, int nx) {
    using namespace wsn;
    const Geo g0 = make_geo(nz, ny, nx), g1 = make_geo(nz / 2, ny / 2, nx / 2), g2 = make_geo(nz / 4, ny / 4, nx / 4);
    const int64_t N0 = g0.vox(), N1 = g1.vox(), N2 = g2.vox();
    const int c0 = n->c[0], c1 = n->c[1], c2 = n->c[2];
    cudaStream_t st = n->stream;
    cudaError_t e = cudaSuccess;
    auto A = [&](const char* name) { return n->buf[name]; };
    auto G = [&](const char* name, int64_t fl) { return buffer(n, std::string("g_") + name, (size_t)(fl * B), &e); };
    float* gY = A("gY");
    float* gA = G("a", 16 * N0 > c2 * N1 ? 32 * N0 : c2 * N1);  // scratch gradients (largest layer)
    float* gB = G("b", 32 * N0);
    float* gL0b = G("L0b", c0 * N0);
    float* gL1b = G("L1b", c1 * N1);
    if (e != cudaSuccess) return wfail(n, LBM_ENOMEM, "gradient buffers: %s", cudaGetErrorString(e));
    auto gw = [&](int k) { return n->g + n->woff[k]; };
    auto gb = [&](int k) { return n->g + n->boff[k]; };
    // conv layer k backward: input activation `in` (cin, geo), output gradient gout (cout)
    auto back = [&](int k, const float* in, const float* gout, float* gin, const Geo& g) -> int {
        const int cout = n->co[k], cin = n->ci[k];
        WS_CUDA(n, conv_bwd_w(cout, in, cin, gout, gw(k), g, B, st));
        k_bias_grad<<<dim3(64, (unsigned)(B * cout)), 256, 0, st>>>(gout, cout, g.vox(), gb(k));
        if (gin) {
            k_flip_weights<<<(cout * cin * 27 + 255) / 256, 256, 0, st>>>(n->p + n->woff[k], cout, cin, n->wt);
            WS_CUDA(n, conv_fwd(cin, gout, cout, n->wt, nullptr, gin, g, B, 0, st));
        }
        return LBM_OK;
    };
    int rc;
    // Y = conv10(L4b) * X  (gY already masked)
    if ((rc = back(10, A("L4b"), gY, gA, g0))) return rc;
    k_relu_mask<<<gs_blocks(B * c0 * N0), 256, 0, st>>>(gA, A("L4b"), (int64_t)B * c0 * N0);
    if ((rc = back(9, A("S0"), gA, gL0b, g0))) return rc;          // gS0 -> gL0b (and gL4a below)
    WS_CUDA(n, cudaMemcpyAsync(gA, gL0b, sizeof(float) * B * c0 * N0, cudaMemcpyDeviceToDevice, st));
    k_relu_mask<<<gs_blocks(B * c0 * N0), 256, 0, st>>>(gA, A("L4a"), (int64_t)B * c0 * N0);
    if ((rc = back(8, A("U0"), gA, gB, g0))) return rc;            // gU0 (c1, N0)
    float* gL3b = G("L3b", c1 * N1);
    if (e != cudaSuccess) return wfail(n, LBM_ENOMEM, "gradient buffers");
    k_up_bwd<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(gB, gL3b, (int64_t)B * c1, g1);
    k_relu_mask<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(gL3b, A("L3b"), (int64_t)B * c1 * N1);
    if ((rc = back(7, A("S1"), gL3b, gL1b, g1))) return rc;        // gS1 -> gL1b (and gL3a)
    WS_CUDA(n, cudaMemcpyAsync(gA, gL1b, sizeof(float) * B * c1 * N1, cudaMemcpyDeviceToDevice, st));
    k_relu_mask<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(gA, A("L3a"), (int64_t)B * c1 * N1);
    if ((rc = back(6, A("U1"), gA, gB, g1))) return rc;            // gU1 (c2, N1)
    float* gL2b = G("L2b", c2 * N2);
    float* gL2a = G("L2a", c2 * N2);
    float* gP2 = G("P2", c1 * N2);
    if (e != cudaSuccess) return wfail(n, LBM_ENOMEM, "gradient buffers");
    k_up_bwd<<<gs_blocks(B * c2 * N2), 256, 0, st>>>(gB, gL2b, (int64_t)B * c2, g2);
    k_relu_mask<<<gs_blocks(B * c2 * N2), 256, 0, st>>>(gL2b, A("L2b"), (int64_t)B * c2 * N2);
    if ((rc = back(5, A("L2a"), gL2b, gL2a, g2))) return rc;
    k_relu_mask<<<gs_blocks(B * c2 * N2), 256, 0, st>>>(gL2a, A("L2a"), (int64_t)B * c2 * N2);
    if ((rc = back(4, A("P2"), gL2a, gP2, g2))) return rc;
    k_pool_bwd<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(gP2, gL1b, (int64_t)B * c1, g1);
    k_relu_mask<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(gL1b, A("L1b"), (int64_t)B * c1 * N1);
    float* gL1a = G("L1a", c1 * N1);
    float* gP1 = G("P1", c0 * N1);
    if (e != cudaSuccess) return wfail(n, LBM_ENOMEM, "gradient buffers");
    if ((rc = back(3, A("L1a"), gL1b, gL1a, g1))) return rc;
    k_relu_mask<<<gs_blocks(B * c1 * N1), 256, 0, st>>>(gL1a, A("L1a"), (int64_t)B * c1 * N1);
    if ((rc = back(2, A("P1"), gL1a, gP1, g1))) return rc;
    k_pool_bwd<<<gs_blocks(B * c0 * N0), 256, 0, st>>>(gP1, gL0b, (int64_t)B * c0, g0);
    k_relu_mask<<<gs_blocks(B * c0 * N0), 256, 0, st>>>(gL0b, A("L0b"), (int64_t)B * c0 * N0);
    if ((rc = back(1, A("L0a"), gL0b, gA, g0))) return rc;
    k_relu_mask<<<gs_blocks(B * c0 * N0), 256, 0, st>>>(gA, A("L0a"), (int64_t)B * c0 * N0);
    if ((rc = back(0, A("X"), gA, nullptr, g0))) return rc;
    WS_CUDA(n, cudaGetLastError());
    return LBM_OK;
}

bool dims_ok(int nz, int ny, int nx) {
    return nz >= 4 && ny >= 4 && nx >= 4 && nz % 4 == 0 && ny % 4 == 0 && nx % 4 == 0;
}

// loss and gradient of B samples already on the device (mask, target)
int loss_grad_dev(lbm_wsnet* n, const uint8_t* d_mask, const float* d_t, int B, int nz, int ny, int nx,
                  double* loss) {
    int rc = forward(n, d_mask, B, nz, ny, nx);
    if (rc) return rc;
    const int64_t N0 = (int64_t)nz * ny * nx;
    cudaError_t e = cudaSuccess;
    float* gY = buffer(n, "gY", (size_t)(B * 3 * N0), &e);
    if (e != cudaSuccess) return wfail(n, LBM_ENOMEM, "gY");
    WS_CUDA(n, cudaMemsetAsync(n->d_cnt, 0, sizeof(unsigned long long), n->stream));
    wsn::k_count<<<wsn::gs_blocks(B * N0), 256, 0, n->stream>>>(n->buf["X"], B * N0, n->d_cnt);
    unsigned long long cnt = 0;
    WS_CUDA(n, cudaMemcpyAsync(&cnt, n->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, n->stream));
    WS_CUDA(n, cudaStreamSynchronize(n->stream));
    if (cnt == 0) return wfail(n, LBM_EINVAL, "no pore voxels");
    WS_CUDA(n, cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream));
    wsn::k_mse<<<wsn::gs_blocks(B * 3 * N0), 256, 0, n->stream>>>(n->buf["Y"], d_t, n->buf["X"], N0, B,
                                                                  1.0 / (3.0 * (double)cnt), gY, n->d_loss);
    WS_CUDA(n, cudaMemsetAsync(n->g, 0, sizeof(float) * n->np, n->stream));
    if ((rc = backward(n, B, nz, ny, nx))) return rc;
    if (loss) {
        WS_CUDA(n, cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        WS_CUDA(n, cudaStreamSynchronize(n->stream));
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_wsnet_create(int c0, int c1, int c2, lbm_wsnet** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    auto okc = [](int c) { return c == 8 || c == 16 || c == 32; };
    if (!okc(c0) || !okc(c1) || !okc(c2)) return LBM_EINVAL;
    auto* n = new (std::nothrow) lbm_wsnet();
    if (!n) return LBM_ENOMEM;
    cudaGetDevice(&n->device);
    n->c[0] = c0;
    n->c[1] = c1;
    n->c[2] = c2;
    const int shp[wsn::kLayers][2] = {{c0, 1}, {c0, c0}, {c1, c0}, {c1, c1}, {c2, c1}, {c2, c2},
                                      {c1, c2}, {c1, c1}, {c0, c1}, {c0, c0}, {3, c0}};
    int64_t k = 0, maxw = 0;
    for (int l = 0; l < wsn::kLayers; ++l) {
        n->co[l] = shp[l][0];
        n->ci[l] = shp[l][1];
        n->woff[l] = k;
        k += (int64_t)n->co[l] * n->ci[l] * 27;
        n->boff[l] = k;
        k += n->co[l];
        maxw = std::max<int64_t>(maxw, (int64_t)n->co[l] * n->ci[l] * 27);
    }
    n->np = k;
    cudaError_t e = cudaMalloc(&n->p, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->g, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->m, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->v, k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->wt, maxw * 4);
    if (e == cudaSuccess) e = cudaMalloc(&n->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&n->d_cnt, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(n->p, 0, k * 4);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, k * 4);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, k * 4);
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
    WS_CUDA(n, cudaMemcpy(n->p, host, n->np * 4, cudaMemcpyHostToDevice));
    WS_CUDA(n, cudaMemset(n->m, 0, n->np * 4));
    WS_CUDA(n, cudaMemset(n->v, 0, n->np * 4));
    n->adam_t = 0;
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
    if (!mask || !target || batch < 1 || !dims_ok(nz, ny, nx))
        return wfail(n, LBM_EINVAL, "bad arguments (sides must be multiples of 4)");
    const int64_t N0 = (int64_t)nz * ny * nx;
    uint8_t* dm = nullptr;
    float* dt = nullptr;
    WS_CUDA(n, cudaMalloc(&dm, batch * N0));
    WS_CUDA(n, cudaMalloc(&dt, batch * 3 * N0 * 4));
    cudaError_t e = cudaMemcpyAsync(dm, mask, batch * N0, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, target, batch * 3 * N0 * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) rc = loss_grad_dev(n, dm, dt, batch, nz, ny, nx, loss);
    if (e == cudaSuccess && rc == LBM_OK && grad) e = cudaMemcpy(grad, n->g, n->np * 4, cudaMemcpyDeviceToHost);
    cudaFree(dm);
    cudaFree(dt);
    if (e != cudaSuccess) return wfail(n, LBM_ECUDA, "lbm_wsnet_loss_grad: %s", cudaGetErrorString(e));
    return rc;
}

int lbm_wsnet_train(lbm_wsnet* n, const uint8_t* masks, const float* targets, int n_samples, int nx, int ny, int nz,
                    int epochs, int batch, float lr, const int* order, float* loss_history) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!masks || !targets || n_samples < 1 || epochs < 1 || batch < 1 || !dims_ok(nz, ny, nx) || !order)
        return wfail(n, LBM_EINVAL, "bad arguments");
    const int64_t N0 = (int64_t)nz * ny * nx;
    uint8_t *dm = nullptr, *bm = nullptr;
    float *dt = nullptr, *bt = nullptr;
    WS_CUDA(n, cudaMalloc(&dm, (size_t)n_samples * N0));
    WS_CUDA(n, cudaMalloc(&dt, (size_t)n_samples * 3 * N0 * 4));
    WS_CUDA(n, cudaMalloc(&bm, (size_t)batch * N0));
    WS_CUDA(n, cudaMalloc(&bt, (size_t)batch * 3 * N0 * 4));
    WS_CUDA(n, cudaMemcpy(dm, masks, (size_t)n_samples * N0, cudaMemcpyHostToDevice));
    WS_CUDA(n, cudaMemcpy(dt, targets, (size_t)n_samples * 3 * N0 * 4, cudaMemcpyHostToDevice));
    for (int ep = 0; ep < epochs && rc == LBM_OK; ++ep) {
        double ep_loss = 0.0;
        int nb = 0;
        for (int s0 = 0; s0 < n_samples && rc == LBM_OK; s0 += batch) {
            const int B = std::min(batch, n_samples - s0);
            for (int j = 0; j < B; ++j) {
                const int idx = order[(size_t)ep * n_samples + s0 + j];
                cudaMemcpyAsync(bm + (size_t)j * N0, dm + (size_t)idx * N0, N0, cudaMemcpyDeviceToDevice, n->stream);
                cudaMemcpyAsync(bt + (size_t)j * 3 * N0, dt + (size_t)idx * 3 * N0, 3 * N0 * 4,
                                cudaMemcpyDeviceToDevice, n->stream);
            }
            double l = 0.0;
            rc = loss_grad_dev(n, bm, bt, B, nz, ny, nx, &l);
            if (rc) break;
            ++n->adam_t;
            const float b1 = 0.9f, b2 = 0.999f;
            wsn::k_adam<<<wsn::gs_blocks(n->np), 256, 0, n->stream>>>(
                n->p, n->g, n->m, n->v, n->np, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)n->adam_t),
                1.f - powf(b2, (float)n->adam_t));
            ep_loss += l;
            ++nb;
        }
        if (loss_history) loss_history[ep] = (float)(ep_loss / std::max(nb, 1));
    }
    cudaError_t e = cudaStreamSynchronize(n->stream);
    cudaFree(dm);
    cudaFree(dt);
    cudaFree(bm);
    cudaFree(bt);
    if (rc) return rc;
    if (e != cudaSuccess) return wfail(n, LBM_ECUDA, "lbm_wsnet_train: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_wsnet_predict(lbm_wsnet* n, const uint8_t* mask, int nx, int ny, int nz, float* y) {
    int rc = wenter(n);
    if (rc) return rc;
    if (!mask || !y || !dims_ok(nz, ny, nx)) return wfail(n, LBM_EINVAL, "bad arguments (sides multiple of 4)");
    const int64_t N0 = (int64_t)nz * ny * nx;
    uint8_t* dm = nullptr;
    WS_CUDA(n, cudaMalloc(&dm, N0));
    cudaError_t e = cudaMemcpyAsync(dm, mask, N0, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) rc = forward(n, dm, 1, nz, ny, nx);
    if (e == cudaSuccess && rc == LBM_OK)
        e = cudaMemcpyAsync(y, n->buf["Y"], 3 * N0 * 4, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    cudaFree(dm);
    if (e != cudaSuccess) return wfail(n, LBM_ECUDA, "lbm_wsnet_predict: %s", cudaGetErrorString(e));
    return rc;
}

int lbm_wsnet_release_buffers(lbm_wsnet* n) {
    int rc = wenter(n);
    if (rc) return rc;
    cudaStreamSynchronize(n->stream);
    for (auto& kv : n->buf) cudaFree(kv.second);
    n->buf.clear();
    n->cap.clear();
    return LBM_OK;
}

int lbm_wsnet_destroy(lbm_wsnet* n) {
    if (!n) return LBM_OK;
    cudaSetDevice(n->device);
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (auto& kv : n->buf) cudaFree(kv.second);
    cudaFree(n->p);
    cudaFree(n->g);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->wt);
    cudaFree(n->d_loss);
    cudaFree(n->d_cnt);
    delete n;
    return LBM_OK;
}

const char* lbm_wsnet_last_error(const lbm_wsnet* n) { return n ? n->err.c_str() : "invalid network handle"; }

}  // extern "C"
