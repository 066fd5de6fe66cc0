// Host runtime and C ABI (include/lbm.h) of the D3Q19 flux-boundary solver.
//
// Geometry is preprocessed once on the host: the pore list in (z, y, x) raster
// order -- so the inlet plane z = 0 holds pore indices [0, A) and the outlet
// plane the last A_out indices -- and a padded int32 id grid whose extra layer
// is SOLID on the lateral faces and ZOUT beyond the z faces, so the kernels
// look up all 18 pull sources without bounds checks.  Distributions are stored
// structure-of-arrays, f[q][i] with row stride ns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <new>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace {

constexpr int kGraphSteps = 64;  // steps per captured graph (even: parity preserved)
#ifndef LBM_DEFAULT_STEP_VARIANT
#define LBM_DEFAULT_STEP_VARIANT 0
#endif
constexpr int kDefaultStepVariant = LBM_DEFAULT_STEP_VARIANT;
constexpr int64_t kReencodeInterval = 1024;  // steps between 16-bit reference refreshes
thread_local std::string g_create_error;

}  // namespace

struct lbm_ctx {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    int model = 1, prec = 1;
    double tau = 1.0;
    lbm::Relax relax{};
    lbm::StepConfig step_cfg{0, 0};
    lbm::DevLattice L{};
    void* f[2] = {nullptr, nullptr};
    int cur = 0;     // buffer of the state (pull variants) and parity of the inlet-density slot
    bool aa = false; // AA pattern: the state lives in f[0] alone, f[1] is released
    // AA pattern: the buffer stays in the in-place layout between lbm_step calls
    // (aa_resident); aa_phase = 0 when the next launch gathers and scatters, 1
    // when it is node-local.  Every other call swaps it back first (aa_settle).
    bool aa_resident = false;
    int aa_phase = 0;
    uint32_t* d_vox = nullptr;
    int* d_grid = nullptr;
    lbm::BcState h_bc{};
    lbm::BcState* d_bc = nullptr;
    double* d_red_partials = nullptr;   // inlet reductions (prime and fused), per-block partials
    unsigned* d_red_counter = nullptr;  // ticket of the stand-alone inlet reduction
    unsigned* d_step_counter = nullptr; // ticket of the reduction fused into the step
    double* d_mon_partials = nullptr;
    unsigned* d_mon_counter = nullptr;
    lbm::MonitorOut* d_mon = nullptr;
    double* d_u_ref = nullptr;  // velocity snapshot of the steady-state criterion (allocated on first use)
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};  // [cur + 2 aa_phase]
    int64_t steps = 0;
    int64_t since_reencode = 0;  // steps since the 16-bit reference profile was refreshed
    int ref_e = 0;               // profile slot the stored values are encoded with
    int status = LBM_OK;
    std::string err;
    std::vector<int64_t> pore_voxel;  // unpadded [z][y][x] index of each pore node
};

namespace {

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (code == LBM_ECUDA) c->status = LBM_ECUDA;
    } else {
        g_create_error = buf;
    }
    return code;
}

#define LBM_CUDA(ctx, call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((ctx), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int aa_settle(lbm_ctx* c);

// True while the context's stream records a CUDA graph.  A failing query (the
// legacy stream while another stream captures globally) counts as not
// capturing; the launches that follow report that case themselves.
bool stream_capturing(lbm_ctx* c) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

// Every entry point but lbm_step: select the device and bring a resident AA
// layout back to the pull layout the other calls read and write.
int enter(lbm_ctx* c, bool settle = true) {
    if (!c) return LBM_EINVAL;
    if (c->status == LBM_ECUDA) return LBM_ECUDA;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return settle ? aa_settle(c) : LBM_OK;
}

// Buffer that holds the current state (pull layout in every variant).
void* state_f(lbm_ctx* c) { return c->aa ? c->f[0] : c->f[c->cur]; }

int push_bc(lbm_ctx* c) {
    // host-owned fields only: the inlet densities, the 16-bit reference profile
    // and the rounding seeds live on the device
    LBM_CUDA(c, cudaMemcpyAsync(c->d_bc, &c->h_bc, lbm::kBcHostBytes, cudaMemcpyHostToDevice, c->stream));
    // h_bc must stay valid until the copy ran: make the copy synchronous w.r.t. the host.
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int one_step(lbm_ctx* c, cudaStream_t st) {
    LBM_CUDA(c, lbm::launch_step_cfg(c->prec, c->step_cfg, state_f(c), c->f[c->cur ^ 1], c->cur, c->L,
                                     c->relax, c->d_bc, c->d_red_partials, c->d_step_counter, st));
    c->cur ^= 1;
    return LBM_OK;
}

// AA pattern, in the in-place layout: a gather-scatter launch when aa_phase is 0,
// a node-local one when it is 1; the two alternate across lbm_step calls.
int aa_step(lbm_ctx* c, cudaStream_t st) {
    LBM_CUDA(c, lbm::launch_aa_step(c->prec, c->f[0], c->aa_phase == 0, c->cur, c->L, c->relax, c->d_bc,
                                    c->d_red_partials, c->d_step_counter, st));
    c->cur ^= 1;
    c->aa_phase ^= 1;
    return LBM_OK;
}

// AA pattern: from the in-place layout back to the pull layout (an un-stream
// swap after a gather-scatter launch, then the opposite-pair swap), on the
// context's stream.  A no-op when the layout is not resident.
int aa_settle_launch(lbm_ctx* c) {
    if (!c->aa_resident) return LBM_OK;
    if (c->aa_phase) LBM_CUDA(c, lbm::launch_aa_unstream(c->prec, c->f[0], c->L, c->d_bc, c->stream));
    LBM_CUDA(c, lbm::launch_aa_swap(c->prec, c->f[0], c->L, c->stream));
    c->aa_resident = false;
    c->aa_phase = 0;
    return LBM_OK;
}

// Host state (buffer parity, layout) advances when a call is made, so a graph
// recorded from the calls must start and end in the pull layout to be replayed.
constexpr const char* kResidentInCapture =
    "the AA-pattern buffer is in its in-place layout while the stream records a graph; "
    "make any other call on the context (e.g. lbm_set_stream) before the capture begins";

int aa_settle(lbm_ctx* c) {
    if (!c->aa_resident) return LBM_OK;
    if (stream_capturing(c)) return fail(c, LBM_EINVAL, "%s", kResidentInCapture);
    return aa_settle_launch(c);
}

// Inlet density for the current buffer when the state or Q changed outside a
// step (steps produce the next density themselves).
int prime_inlet(lbm_ctx* c) {
    LBM_CUDA(c, lbm::launch_inlet_reduce(c->prec, state_f(c), c->cur, c->L, c->d_bc, c->d_red_partials,
                                         c->d_red_counter, c->stream));
    return LBM_OK;
}

// 16-bit formats: refresh the reference density profile (re-encoding the
// state) every kReencodeInterval steps, then recompute the inlet density from
// the re-encoded values.  Asynchronous; a no-op for FP32/FP64.
int maybe_reencode(lbm_ctx* c) {
    if (c->prec < LBM_PREC_FP16DEV || c->since_reencode < kReencodeInterval) return LBM_OK;
    LBM_CUDA(c, lbm::launch_reencode(c->prec, state_f(c), c->L, c->d_bc, c->ref_e, c->cur, c->stream));
    c->ref_e ^= 1;
    c->since_reencode = 0;
    return prime_inlet(c);
}

// Graph slot gi = cur + 2 aa_phase: kGraphSteps steps starting from that buffer
// parity (and, on the AA pattern, that launch kind).
int build_graph(lbm_ctx* c, int gi) {
    static_assert(kGraphSteps % 2 == 0, "a graph must preserve the buffer parity and the AA phase");
    const int saved = c->cur, saved_phase = c->aa_phase;
    c->cur = gi & 1;
    c->aa_phase = gi >> 1;
    cudaGraph_t g = nullptr;
    LBM_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    for (int k = 0; k < kGraphSteps && rc == LBM_OK; ++k) rc = c->aa ? aa_step(c, c->cap_stream) : one_step(c, c->cap_stream);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->cur = saved;
    c->aa_phase = saved_phase;
    if (rc != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph[gi], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int run_monitors(lbm_ctx* c, lbm::MonitorOut* out) {
    LBM_CUDA(c, lbm::launch_monitors(c->prec, state_f(c), c->L, c->d_bc, c->d_mon_partials, c->d_mon_counter,
                                     c->d_mon, c->stream));
    LBM_CUDA(c, cudaMemcpyAsync(out, c->d_mon, sizeof(*out), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

void release(lbm_ctx* c) {
    for (auto& g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto& p : c->f)
        if (p) cudaFree(p);
    cudaFree(c->d_vox);
    cudaFree(c->d_grid);
    cudaFree(c->d_bc);
    cudaFree(c->d_red_partials);
    cudaFree(c->d_red_counter);
    cudaFree(c->d_step_counter);
    cudaFree(c->d_mon_partials);
    cudaFree(c->d_mon_counter);
    cudaFree(c->d_mon);
    cudaFree(c->d_u_ref);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
}

template <class T>
int dev_alloc(lbm_ctx* c, T** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "cudaMalloc(%zu): %s",
                    bytes, cudaGetErrorString(e));
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_create(const uint8_t* mask, int nx, int ny, int nz, double tau, int model, int precision,
               lbm_ctx** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mask) return fail(nullptr, LBM_EINVAL, "mask is NULL");
    if (nx < 1 || ny < 1 || nx > 2047 || ny > 2047 || nz < 3 || nz > 1023)
        return fail(nullptr, LBM_EINVAL, "box %dx%dx%d outside 1..2047 x 1..2047 x 3..1023", nx, ny, nz);
    if (!(tau > 0.5) || !(tau < 1e6)) return fail(nullptr, LBM_EINVAL, "tau=%g must exceed 0.5", tau);
    if (model != LBM_MODEL_BGK && model != LBM_MODEL_MRT)
        return fail(nullptr, LBM_EINVAL, "unknown model %d", model);
    if (precision < LBM_PREC_FP64 || precision > LBM_PREC_BF16DEV)
        return fail(nullptr, LBM_EINVAL, "unknown precision %d", precision);
    const int64_t px = nx + 2, py = ny + 2, pz = nz + 2;
    if (px * py * pz > (int64_t)UINT32_MAX)
        return fail(nullptr, LBM_EINVAL, "padded box exceeds 2^32 voxels");
    const int64_t ncell = (int64_t)nx * ny * nz;

    auto* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation");
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->model = model;
    c->prec = precision;
    c->tau = tau;
    {
        const double sp = 1.0 / tau;
        c->relax.sp = sp;
        c->relax.sm = model == LBM_MODEL_MRT ? 8.0 * (2.0 - sp) / (8.0 - sp) : sp;
    }
    cudaGetDevice(&c->device);

    // ---- pore list, padded id grid (host)
    std::vector<int> grid((size_t)(px * py * pz), lbm::SOLID);
    for (int64_t y = 0; y < py; ++y)
        for (int64_t x = 0; x < px; ++x) {
            grid[(size_t)((0 * py + y) * px + x)] = lbm::ZOUT;
            grid[(size_t)(((pz - 1) * py + y) * px + x)] = lbm::ZOUT;
        }
    std::vector<uint32_t> vox;
    vox.reserve((size_t)(ncell / 2 + 16));
    c->pore_voxel.reserve((size_t)(ncell / 2 + 16));
    int64_t a_in = 0, a_out = 0, a_01 = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t v = (z * ny + y) * nx + x;
                const uint8_t m = mask[v];
                if (m > 1) {
                    delete c;
                    return fail(nullptr, LBM_EINVAL, "mask value %d at voxel %lld (must be 0 or 1)", m,
                                (long long)v);
                }
                if (m) continue;
                const int64_t id = (int64_t)vox.size();
                if (id >= INT32_MAX) {
                    delete c;
                    return fail(nullptr, LBM_EINVAL, "more than 2^31-1 pore nodes");
                }
                const int64_t p = ((z + 1) * py + (y + 1)) * px + (x + 1);
                grid[(size_t)p] = (int)id;
                vox.push_back((uint32_t)p);
                c->pore_voxel.push_back(v);
                if (z == 0) ++a_in;
                if (z <= 1) ++a_01;
                if (z == nz - 1) ++a_out;
            }
    if (a_in == 0 || a_out == 0) {
        delete c;
        return fail(nullptr, LBM_EINVAL, "inlet (%lld) and outlet (%lld) planes need pore nodes",
                    (long long)a_in, (long long)a_out);
    }
    const int64_t n = (int64_t)vox.size();
    c->L.n = n;
    c->L.ns = (n + 127) / 128 * 128;
    c->L.a_in = a_in;
    c->L.a_out = a_out;
    c->L.a_01 = a_01;
    c->L.nx = nx;
    c->L.ny = ny;
    c->L.nz = nz;
    c->L.sy = (int)px;
    c->L.sz = (int)(px * py);
    for (int q = 0; q < 19; ++q)
        c->L.goff[q] = -(lbm::cz(q) * c->L.sz + lbm::cy(q) * c->L.sy + lbm::cx(q));
    {
        const unsigned __int128 two64 = (unsigned __int128)1 << 64;
        const unsigned __int128 szq = (unsigned __int128)(uint64_t)c->L.sz;
        c->L.sz_magic = (uint64_t)(two64 / szq + (two64 % szq != 0 ? 1 : 0));
    }

    // ---- device memory
    int rc = LBM_OK;
    const size_t fbytes = (size_t)19 * (size_t)c->L.ns * (size_t)lbm::elem_size(precision);
    // per-tile partials of the inlet reductions (tiles of >= 128 nodes)
    const int nb_red = std::max(lbm::inlet_reduce_blocks(c->L), (int)((a_01 + 127) / 128));
    const int nb_mon = lbm::monitor_blocks(c->L);
    if ((rc = dev_alloc(c, &c->f[0], fbytes)) || (rc = dev_alloc(c, &c->f[1], fbytes)) ||
        (rc = dev_alloc(c, &c->d_vox, vox.size() * sizeof(uint32_t))) ||
        (rc = dev_alloc(c, &c->d_grid, grid.size() * sizeof(int))) ||
        (rc = dev_alloc(c, &c->d_bc, sizeof(lbm::BcState))) ||
        (rc = dev_alloc(c, &c->d_red_partials, (size_t)nb_red * sizeof(double))) ||
        (rc = dev_alloc(c, &c->d_red_counter, sizeof(unsigned))) ||
        (rc = dev_alloc(c, &c->d_step_counter, sizeof(unsigned))) ||
        (rc = dev_alloc(c, &c->d_mon_partials, (size_t)5 * nb_mon * sizeof(double))) ||
        (rc = dev_alloc(c, &c->d_mon_counter, sizeof(unsigned))) ||
        (rc = dev_alloc(c, &c->d_mon, sizeof(lbm::MonitorOut)))) {
        g_create_error = c->err;
        release(c);
        delete c;
        return rc;
    }
    c->L.vox = c->d_vox;
    c->L.grid = c->d_grid;
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_vox, vox.data(), vox.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_grid, grid.data(), grid.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_red_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_step_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_mon_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->f[0], 0, fbytes);
    if (e == cudaSuccess) e = cudaMemset(c->f[1], 0, fbytes);
    c->h_bc = lbm::BcState{};
    if (e == cudaSuccess) e = cudaMemcpy(c->d_bc, &c->h_bc, sizeof(lbm::BcState), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = lbm::launch_init_eq(precision, c->f[0], c->L, c->d_bc, nullptr, nullptr, nullptr, nullptr, 0);
    if (e == cudaSuccess)
        e = lbm::launch_inlet_reduce(precision, c->f[0], 0, c->L, c->d_bc, c->d_red_partials, c->d_red_counter, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = lbm::configure_step(precision, kDefaultStepVariant, c->L, &c->step_cfg);
    if (e != cudaSuccess) {
        fail(nullptr, LBM_ECUDA, "lbm_create device setup: %s", cudaGetErrorString(e));
        release(c);
        delete c;
        return LBM_ECUDA;
    }
    *out = c;
    return LBM_OK;
}

int lbm_set_flux_bc(lbm_ctx* c, int face, double Q) {
    int rc = enter(c);
    if (rc) return rc;
    if (face == LBM_FACE_ZMAX)
        return fail(c, LBM_EUNSUPPORTED, "flux condition only at the inlet (LBM_FACE_ZMIN)");
    if (face != LBM_FACE_ZMIN) return fail(c, LBM_EINVAL, "unknown face %d", face);
    if (!(Q == Q) || Q > 1e30 || Q < -1e30) return fail(c, LBM_EINVAL, "Q must be finite");
    c->h_bc.Q = Q;
    c->h_bc.inlet_mode = 0;
    if ((rc = push_bc(c))) return rc;
    return prime_inlet(c);
}

int lbm_set_pressure_bc(lbm_ctx* c, int face, double rho) {
    int rc = enter(c);
    if (rc) return rc;
    if (!(rho > 0.0) || rho > 1e30) return fail(c, LBM_EINVAL, "rho must be positive and finite");
    if (face == LBM_FACE_ZMAX) {
        c->h_bc.drho_out = rho - 1.0;
    } else if (face == LBM_FACE_ZMIN) {
        c->h_bc.drho_in_fixed = rho - 1.0;
        c->h_bc.inlet_mode = 1;
    } else {
        return fail(c, LBM_EINVAL, "unknown face %d", face);
    }
    if ((rc = push_bc(c))) return rc;
    return prime_inlet(c);
}

int lbm_set_stream(lbm_ctx* c, void* s) {
    int rc = enter(c);
    if (rc) return rc;
    c->stream = (cudaStream_t)s;
    return LBM_OK;
}

int lbm_set_kernel(lbm_ctx* c, int variant) {
    int rc = enter(c);
    if (rc) return rc;
    if (variant < 0 || variant > 3) return fail(c, LBM_EINVAL, "unknown step kernel variant %d", variant);
    lbm::StepConfig cfg{};
    if (variant < 3) LBM_CUDA(c, lbm::configure_step(c->prec, variant, c->L, &cfg));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (variant == 3 && !c->aa) {
        // keep the state buffer as f[0] (cur stays the inlet-density slot) and release the other
        if (c->cur == 1) std::swap(c->f[0], c->f[1]);
        LBM_CUDA(c, cudaFree(c->f[1]));
        c->f[1] = nullptr;
        c->aa = true;
    } else if (variant < 3 && c->aa) {
        const size_t fbytes = (size_t)19 * (size_t)c->L.ns * (size_t)lbm::elem_size(c->prec);
        if ((rc = dev_alloc(c, &c->f[1], fbytes))) return rc;
        if (c->cur == 1) std::swap(c->f[0], c->f[1]);  // the state must sit in f[cur]
        c->aa = false;
    }
    c->step_cfg = cfg;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int n) {
    int rc = enter(c, false);
    if (rc) return rc;
    if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
    if (n == 0) return LBM_OK;
    if (c->aa) {
        // The buffer enters the in-place layout once and stays in it across
        // calls; segments end where the 16-bit reference profile is refreshed,
        // which works on the pull layout.  A call recorded into a graph starts
        // and ends in the pull layout instead.
        const bool capturing = stream_capturing(c);
        if (capturing && c->aa_resident) return fail(c, LBM_EINVAL, "%s", kResidentInCapture);
        int64_t done = 0;
        while (done < n) {
            if (c->prec >= LBM_PREC_FP16DEV && c->since_reencode >= kReencodeInterval) {
                if ((rc = aa_settle_launch(c)) || (rc = maybe_reencode(c))) return rc;
            }
            int64_t seg = n - done;
            if (c->prec >= LBM_PREC_FP16DEV) seg = std::min<int64_t>(seg, kReencodeInterval - c->since_reencode);
            if (!c->aa_resident) {
                LBM_CUDA(c, lbm::launch_aa_swap(c->prec, c->f[0], c->L, c->stream));
                c->aa_resident = true;
                c->aa_phase = 0;
            }
            int64_t k = 0;
            while (seg - k >= kGraphSteps) {
                const int gi = c->cur + 2 * c->aa_phase;
                if (!c->graph[gi] && (rc = build_graph(c, gi))) return rc;
                LBM_CUDA(c, cudaGraphLaunch(c->graph[gi], c->stream));
                k += kGraphSteps;
            }
            for (; k < seg; ++k)
                if ((rc = aa_step(c, c->stream))) return rc;
            done += seg;
            c->since_reencode += seg;
        }
        if (capturing && (rc = aa_settle_launch(c))) return rc;
        c->steps += n;
        return LBM_OK;
    }
    int k = 0;
    while (n - k >= kGraphSteps) {
        if ((rc = maybe_reencode(c))) return rc;
        if (!c->graph[c->cur] && (rc = build_graph(c, c->cur))) return rc;
        LBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
        k += kGraphSteps;
        c->since_reencode += kGraphSteps;
    }
    for (; k < n; ++k) {
        if ((rc = maybe_reencode(c))) return rc;
        if ((rc = one_step(c, c->stream))) return rc;
        ++c->since_reencode;
    }
    c->steps += n;
    return LBM_OK;
}

int lbm_time_kernels(lbm_ctx* c, int n, float* ms_step, float* ms_inlet) {
    int rc = enter(c);
    if (rc) return rc;
    if (n < 1) return fail(c, LBM_EINVAL, "n must be >= 1");
    std::vector<cudaEvent_t> ev((size_t)2 * n, nullptr);
    for (auto& e : ev) LBM_CUDA(c, cudaEventCreate(&e));
    if (c->aa) LBM_CUDA(c, lbm::launch_aa_swap(c->prec, c->f[0], c->L, c->stream));
    for (int k = 0; k < n; ++k) {
        LBM_CUDA(c, cudaEventRecord(ev[2 * k], c->stream));
        if (c->aa) {
            LBM_CUDA(c, lbm::launch_aa_step(c->prec, c->f[0], (k & 1) == 0, c->cur, c->L, c->relax, c->d_bc,
                                            c->d_red_partials, c->d_step_counter, c->stream));
        } else {
            LBM_CUDA(c, lbm::launch_step_cfg(c->prec, c->step_cfg, state_f(c), c->f[c->cur ^ 1], c->cur, c->L,
                                             c->relax, c->d_bc, c->d_red_partials, c->d_step_counter, c->stream));
        }
        LBM_CUDA(c, cudaEventRecord(ev[2 * k + 1], c->stream));
        c->cur ^= 1;
    }
    if (c->aa) {
        if (n & 1) LBM_CUDA(c, lbm::launch_aa_unstream(c->prec, c->f[0], c->L, c->d_bc, c->stream));
        LBM_CUDA(c, lbm::launch_aa_swap(c->prec, c->f[0], c->L, c->stream));
    }
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    double t_st = 0.0;
    for (int k = 0; k < n; ++k) {
        float b = 0.f;
        LBM_CUDA(c, cudaEventElapsedTime(&b, ev[2 * k], ev[2 * k + 1]));
        t_st += b;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    c->steps += n;
    if (ms_step) *ms_step = (float)(t_st / n);
    if (ms_inlet) *ms_inlet = 0.0f;  // the inlet reduction runs inside the step kernel
    return LBM_OK;
}

int lbm_get_monitors(lbm_ctx* c, double* mass, double* q_in, double* q_out, double* u_max) {
    int rc = enter(c);
    if (rc) return rc;
    lbm::MonitorOut m{};
    if ((rc = run_monitors(c, &m))) return rc;
    if (mass) *mass = (double)c->L.n + m.drho_sum;
    if (q_in) *q_in = m.q_in;
    if (q_out) *q_out = m.q_out;
    const double um = m.umax2 >= 0 ? std::sqrt(m.umax2) : m.umax2;
    if (u_max) *u_max = um;
    if (m.nan_count > 0 || !(um <= 0.1) || !(m.drho_sum == m.drho_sum))
        return fail(c, LBM_EUNSTABLE, "unstable state: %g non-finite nodes, max|u| = %g", m.nan_count, um);
    return LBM_OK;
}

int lbm_steady_residual(lbm_ctx* c, double* residual) {
    int rc = enter(c);
    if (rc) return rc;
    if (!residual) return fail(c, LBM_EINVAL, "residual is NULL");
    const bool first = c->d_u_ref == nullptr;
    if (first) {
        if ((rc = dev_alloc(c, &c->d_u_ref, (size_t)3 * c->L.n * sizeof(double)))) return rc;
        LBM_CUDA(c, cudaMemsetAsync(c->d_u_ref, 0, (size_t)3 * c->L.n * sizeof(double), c->stream));
    }
    LBM_CUDA(c, lbm::launch_velocity_change(c->prec, state_f(c), c->L, c->d_bc, c->d_u_ref, c->d_mon_partials,
                                            c->d_mon_counter, c->d_mon, c->stream));
    lbm::MonitorOut m{};
    LBM_CUDA(c, cudaMemcpyAsync(&m, c->d_mon, sizeof m, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (first)
        *residual = HUGE_VAL;
    else
        *residual = m.q_in > 0.0 ? m.drho_sum / m.q_in : (m.drho_sum > 0.0 ? HUGE_VAL : 0.0);
    return LBM_OK;
}

int lbm_get_flux(lbm_ctx* c, int face, double* Q, double* rho_bc) {
    int rc = enter(c);
    if (rc) return rc;
    if (face != LBM_FACE_ZMIN && face != LBM_FACE_ZMAX) return fail(c, LBM_EINVAL, "unknown face %d", face);
    lbm::MonitorOut m{};
    if ((rc = run_monitors(c, &m))) return rc;
    lbm::BcState b{};
    LBM_CUDA(c, cudaMemcpy(&b, c->d_bc, sizeof b, cudaMemcpyDeviceToHost));
    if (Q) *Q = face == LBM_FACE_ZMIN ? m.q_in : m.q_out;
    if (rho_bc)
        *rho_bc = 1.0 + (face == LBM_FACE_ZMAX ? b.drho_out
                         : b.inlet_mode        ? b.drho_in_fixed
                                               : b.drho_in[c->cur ^ 1]);
    return LBM_OK;
}

int lbm_get_fields(lbm_ctx* c, double* rho, double* ux, double* uy, double* uz) {
    int rc = enter(c);
    if (rc) return rc;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    double* d = nullptr;
    if ((rc = dev_alloc(c, &d, 4 * ncell * sizeof(double)))) return rc;
    double* outs[4] = {rho, ux, uy, uz};
    cudaError_t e = cudaMemsetAsync(d, 0, 4 * ncell * sizeof(double), c->stream);
    if (e == cudaSuccess)
        e = lbm::launch_export(c->prec, state_f(c), c->L, c->d_bc, d, d + ncell, d + 2 * ncell, d + 3 * ncell, 1,
                               c->stream);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (outs[k])
            e = cudaMemcpyAsync(outs[k], d + k * ncell, ncell * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "lbm_get_fields: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_get_fields_device(lbm_ctx* c, float* rho, float* u) {
    int rc = enter(c);
    if (rc) return rc;
    if (!rho && !u) return LBM_OK;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    if (rho) LBM_CUDA(c, cudaMemsetAsync(rho, 0, ncell * sizeof(float), c->stream));
    if (u) LBM_CUDA(c, cudaMemsetAsync(u, 0, 3 * ncell * sizeof(float), c->stream));
    LBM_CUDA(c, lbm::launch_export(c->prec, state_f(c), c->L, c->d_bc, rho, u, u ? u + ncell : nullptr,
                                   u ? u + 2 * ncell : nullptr, 0, c->stream));
    return LBM_OK;
}

int lbm_set_fields(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* uz) {
    int rc = enter(c);
    if (rc) return rc;
    const int64_t n = c->L.n;
    const double* ins[4] = {rho, ux, uy, uz};
    std::vector<double> h((size_t)(4 * n));
    for (int k = 0; k < 4; ++k)
        if (ins[k])
            for (int64_t i = 0; i < n; ++i) h[(size_t)(k * n + i)] = ins[k][c->pore_voxel[(size_t)i]];
    double* d = nullptr;
    if ((rc = dev_alloc(c, &d, h.size() * sizeof(double)))) return rc;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = lbm::launch_init_eq(c->prec, state_f(c), c->L, c->d_bc, rho ? d : nullptr, ux ? d + n : nullptr,
                                uy ? d + 2 * n : nullptr, uz ? d + 3 * n : nullptr, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "lbm_set_fields: %s", cudaGetErrorString(e));
    c->steps = 0;
    return prime_inlet(c);
}

int lbm_get_distributions(lbm_ctx* c, double* f) {
    int rc = enter(c);
    if (rc) return rc;
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    const int64_t n = c->L.n;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    std::vector<double> h((size_t)(19 * n));
    double* d = nullptr;
    if ((rc = dev_alloc(c, &d, h.size() * sizeof(double)))) return rc;
    cudaError_t e = lbm::launch_decode(c->prec, state_f(c), c->L, c->d_bc, d, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "lbm_get_distributions: %s", cudaGetErrorString(e));
    std::memset(f, 0, 19 * ncell * sizeof(double));
    for (int q = 0; q < 19; ++q) {
        const double w = lbm::wq(q);
        for (int64_t i = 0; i < n; ++i)
            f[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]] = w + h[(size_t)(q * n + i)];
    }
    return LBM_OK;
}

int lbm_set_distributions(lbm_ctx* c, const double* f) {
    int rc = enter(c);
    if (rc) return rc;
    if (!f) return fail(c, LBM_EINVAL, "f is NULL");
    const int64_t n = c->L.n;
    const size_t ncell = (size_t)c->nx * c->ny * c->nz;
    std::vector<double> h((size_t)(19 * n));
    for (int q = 0; q < 19; ++q) {
        const double w = lbm::wq(q);
        for (int64_t i = 0; i < n; ++i)
            h[(size_t)(q * n + i)] = f[(size_t)q * ncell + (size_t)c->pore_voxel[(size_t)i]] - w;
    }
    double* d = nullptr;
    if ((rc = dev_alloc(c, &d, h.size() * sizeof(double)))) return rc;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = lbm::launch_encode(c->prec, state_f(c), c->L, c->d_bc, d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "lbm_set_distributions: %s", cudaGetErrorString(e));
    c->steps = 0;
    return prime_inlet(c);
}

int lbm_get_info(const lbm_ctx* c, int64_t* n_pore, int64_t* a_in, int64_t* a_out, int64_t* steps) {
    if (!c) return LBM_EINVAL;
    if (n_pore) *n_pore = c->L.n;
    if (a_in) *a_in = c->L.a_in;
    if (a_out) *a_out = c->L.a_out;
    if (steps) *steps = c->steps;
    return LBM_OK;
}

int lbm_inlet_density_noalloc(lbm_ctx* c, double* rho_in_device) {
    int rc = enter(c);
    if (rc) return rc;
    if (!rho_in_device) return fail(c, LBM_EINVAL, "rho_in_device is NULL");
    if (c->L.a_in > lbm::noalloc_max_inlet_nodes())
        return fail(c, LBM_EINVAL,
                    "inlet has %lld pore nodes; lbm_inlet_density_noalloc supports at most %lld",
                    (long long)c->L.a_in, (long long)lbm::noalloc_max_inlet_nodes());
    LBM_CUDA(c, lbm::launch_inlet_density_noalloc(c->prec, state_f(c), c->L, c->d_bc, rho_in_device,
                                                  c->stream));
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
