// Internal interface between the C-ABI layer (lbm_api.cu) and the kernels
// (lbm_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace lbm {

struct BcState;

// Geometry of one lattice on the device.
struct DevLattice {
    int64_t n;          // pore nodes
    int64_t ns;         // row stride of the distribution arrays (elements)
    int64_t a_in;       // inlet pore nodes: pore indices [0, a_in)
    int64_t a_out;      // outlet pore nodes: pore indices [n - a_out, n)
    int64_t a_01;       // pore nodes on the planes z = 0 and z = 1: indices [0, a_01)
    int nx, ny, nz;     // voxel box
    int sy, sz;         // strides of the padded id grid: (nx+2), (nx+2)(ny+2)
    const uint32_t* vox;  // [n] padded linear voxel index of each pore node
    const int* grid;      // [(nz+2)(ny+2)(nx+2)] padded id grid
    int goff[19];         // padded-grid offset of the pull source x - xi_q, per q
    uint64_t sz_magic;    // ceil(2^64 / sz): plane of a padded voxel index
};

struct Relax {
    double sp, sm;  // s+ and s- of the two-relaxation-time form
};

// Monitor outputs (device), reduced in fixed order.
struct MonitorOut {
    double drho_sum;  // sum of (rho - 1) over pore nodes
    double q_in;      // sum of u_z over inlet pore nodes
    double q_out;     // sum of u_z over outlet pore nodes
    double umax2;     // max |u|^2
    double nan_count; // number of pore nodes with a non-finite moment
};

// Launchers.  `prec` is the LBM_PREC_* code.  All are asynchronous on `st`.
// Inlet density of Eq. (potential) for buffer `fin` (parity `slot`) by a pull
// over the inlet plane; used whenever the state or Q changes outside a step.
cudaError_t launch_inlet_reduce(int prec, const void* fin, int slot, const DevLattice& L, BcState* bc,
                                double* partials, unsigned* counter, cudaStream_t st);
// One full step fin (parity `slot`) -> fout; also produces drho_in[slot ^ 1].
cudaError_t launch_step(int prec, const void* fin, void* fout, int slot, const DevLattice& L, Relax r,
                        BcState* bc, double* partials, unsigned* counter, cudaStream_t st);
int step_reduce_blocks(const DevLattice& L);

// Step-kernel variant: 0 = one thread per node (k_step); 1 / 2 = persistent
// cp.async-pipelined kernel (k_step_async) with 256 / 128-node tiles.
struct StepConfig {
    int variant;
    int grid;  // persistent grid size of the pipelined kernel
};
cudaError_t configure_step(int prec, int variant, const DevLattice& L, StepConfig* cfg);
cudaError_t launch_step_cfg(int prec, const StepConfig& cfg, const void* fin, void* fout, int slot,
                            const DevLattice& L, Relax r, BcState* bc, double* partials, unsigned* counter,
                            cudaStream_t st);
// AA pattern (single buffer): one odd (gather-scatter) or even
// (node-local) step in place, and the layout swaps around a call.
cudaError_t launch_aa_step(int prec, void* f, int odd, int slot, const DevLattice& L, Relax r, BcState* bc,
                           double* partials, unsigned* counter, cudaStream_t st);
cudaError_t launch_aa_swap(int prec, void* f, const DevLattice& L, cudaStream_t st);
cudaError_t launch_aa_unstream(int prec, void* f, const DevLattice& L, const BcState* bc, cudaStream_t st);
cudaError_t launch_monitors(int prec, const void* f, const DevLattice& L, const BcState* bc, double* partials,
                            unsigned* counter, MonitorOut* out, cudaStream_t st);
cudaError_t launch_velocity_change(int prec, const void* f, const DevLattice& L, const BcState* bc, double* u_ref,
                                   double* partials, unsigned* counter, MonitorOut* out, cudaStream_t st);
cudaError_t launch_export(int prec, const void* f, const DevLattice& L, const BcState* bc, void* rho, void* ux,
                          void* uy, void* uz, int out_double, cudaStream_t st);
cudaError_t launch_init_eq(int prec, void* f, const DevLattice& L, const BcState* bc, const double* rho,
                           const double* ux, const double* uy, const double* uz, cudaStream_t st);
cudaError_t launch_encode(int prec, void* f, const DevLattice& L, const BcState* bc, const double* d,
                          cudaStream_t st);
cudaError_t launch_decode(int prec, const void* f, const DevLattice& L, const BcState* bc, double* d,
                          cudaStream_t st);
// 16-bit formats: move the stored values to a new reference profile (no-op otherwise).
cudaError_t launch_reencode(int prec, void* f, const DevLattice& L, BcState* bc, int e, int slot,
                            cudaStream_t st);

// No-allocation inlet density (lbm_noalloc.cu): scratch in a static device array.
cudaError_t launch_inlet_density_noalloc(int prec, const void* fin, const DevLattice& L,
                                         const BcState* bc, double* rho_in_out, cudaStream_t st);
int64_t noalloc_max_inlet_nodes();

int elem_size(int prec);
int inlet_reduce_blocks(const DevLattice& L);
int monitor_blocks(const DevLattice& L);

}  // namespace lbm
