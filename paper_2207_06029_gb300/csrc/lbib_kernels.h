// Host-side launchers of the liblbib kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbib_device.cuh"

namespace lbib {

// Launches a kernel of the step chain with programmatic stream
// serialization: its blocks may be scheduled while the previous kernel in
// the stream ends, and wait in chain_wait() for that kernel's results
// (this hides the launch gap between the short kernels of the IB stage).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// sweep.cu
// part: 0 the whole lattice, 1 the nodes outside box, 2 the nodes inside box
// stamp == nullptr: no IB force is read; step points to the device step counter
// sr: the lattice's two-word rounding-seed counter, parity: the step's parity
cudaError_t launch_sweep(int prec, const void *fin, void *fout, void *force, const uint32_t *stamp,
                         const uint32_t *step, const Lattice &L, void *fields, int part, const int *box,
                         uint32_t *sr, int parity, int nsm, cudaStream_t s);
cudaError_t prepare_sweep_kernels();
// global mass and momentum (FP64): part holds totals_scratch_doubles() doubles,
// count one word that starts (and is left) at zero, out 4 doubles
cudaError_t launch_totals(int prec, const void *fin, const Lattice &L, double *part, unsigned int *count,
                          double *out, cudaStream_t s);
int totals_scratch_doubles();
// divergence watchdog: part and count as for launch_totals (shared with it,
// same stream), w 2 doubles (reference mass, last mass), err the context's
// error word
cudaError_t launch_watch(int prec, const void *fin, const Lattice &L, double *part, unsigned int *count, double *w,
                         double tol, int *err, cudaStream_t s);
// rho and u null: density 1 and u_x = shear_lo + (shear_hi - shear_lo) z / (nz - 1)
cudaError_t launch_init_equilibrium(int prec, void *fout, const Lattice &L, const double *rho, const double *u,
                                    void *fields, cudaStream_t s, double shear_lo = 0.0, double shear_hi = 0.0);
cudaError_t launch_pop_to_aos(int prec, const void *fin, const Lattice &L, double *out, cudaStream_t s);
cudaError_t launch_aos_to_pop(int prec, const double *in, const Lattice &L, void *fout, cudaStream_t s);
cudaError_t launch_fields_out(int prec, const void *fields, const Lattice &L, double *rho, double *u,
                              cudaStream_t s);

// ib.cu
int mls_blocks(const BodyView &B);
cudaError_t prepare_kernels();
// step_inc: device step counter incremented at the start of the step (first
// body only), or nullptr.  grid_cap > 0: the MLS, structure and spreading
// kernels launch at most grid_cap blocks, each taking its share of their
// blocks' work in turn (0: their full grids)
cudaError_t launch_ib_front(int prec, const void *fin, const Lattice &L, const BodyView &B, void *mom, int nsm,
                            int *err, uint32_t *step_inc, int grid_cap, cudaStream_t s);
cudaError_t launch_membrane(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                            const uint32_t *step, int grid_cap, cudaStream_t s);
cudaError_t launch_rigid(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                         const uint32_t *step, int grid_cap, cudaStream_t s);

// batches (sweep.cu and ib.cu); grid sizes are the totals of the prefix tables
struct BatchGrid {
    int sweep, mom, mls, memb, rf, rm, cen;
};
cudaError_t launch_batch_ib(int prec, const BatchTables &T, const BatchGrid &G, int phase, cudaStream_t s);
cudaError_t launch_batch_sweep(int prec, const BatchTables &T, const BatchGrid &G, int phase, int store_fields,
                               cudaStream_t s);
// persistent batched step (ib.cu): P.nsteps steps of every lattice in one
// launch of `grid` blocks of 256 threads; the counters P.ticket, P.abort and
// P.done must be zero at launch
cudaError_t launch_batch_persistent(int prec, const BatchTables &T, const PersistTables &P, int grid, cudaStream_t s);
// resident blocks per SM of the persistent kernel (sets its shared-memory
// attribute; call before any capture)
int batch_persistent_blocks_per_sm(int prec, bool off32);

}  // namespace lbib
