// pt_kernels.h -- launchers of the sm_103a kernels (library-private).
#pragma once
#include <cuda_runtime.h>

#include "pt_internal.h"

namespace ptg {

// Largest dynamic shared memory a sweep-kernel CTA may request on the current device.
cudaError_t sweep_smem_capacity(int* bytes);
cudaError_t set_sweep_smem_limit(int bytes);
// Resident sweep-kernel CTAs per SM for a block size and dynamic shared memory.
cudaError_t sweep_occupancy(int block, int smem_bytes, int* blocks_per_sm, bool slot_major = false,
                            bool walk = false);
cudaError_t launch_init(const InstDesc* insts, const int2* items, int nitems, bool draw,
                        cudaStream_t st);
cudaError_t launch_energy(const InstDesc* insts, const int2* items, int nitems, int32_t first_value,
                          cudaStream_t st);
// mode 0: nsweeps sweeps s = sweep0+1..; mode 1: one exchange sweep with counter sweep0.
// slot_major: every bundle uses the slot-major mapping (Bundle::team > 0),
// otherwise the cell-major one (Bundle::team == 0).  walk: the instances carry
// walk arrays (InstDesc::whot, wtrips, wstate) and the launch updates them.
// L: the lattice side of every instance in the launch (0 if unknown or mixed);
// both slot-major kernels (walk tracked or not) have instantiations for
// L = 4, 8, 12 and 16 with the side as a compile-time constant.
cudaError_t launch_sweeps(const InstDesc* insts, const Bundle* bundles, int nbundles, int grid,
                          int block, int smem_bytes, uint32_t sweep0, int nsweeps, int xevery,
                          int mode, int* queue, cudaStream_t st, bool slot_major = false,
                          bool walk = false, int L = 0);
// dist [n][n]: spins differing between sampled configurations of instance 0
// (sample k: run run[k], slot slot[k]; device arrays).
cudaError_t launch_hamming(const InstDesc* insts, int n, const int32_t* run, const int32_t* slot, int32_t* dist,
                           cudaStream_t st);
// targets (device, one per instance, may be NULL): per-instance target
// energies instead of `target`.
cudaError_t launch_tts(const InstDesc* insts, int ninst, int32_t target, int32_t horizon,
                       int32_t* out, cudaStream_t st, const int32_t* targets = nullptr);

// Debug builds (-DPT_DEBUG): the kernels check their data-dependent indexes
// and record the first failure in a device word.  debug_check synchronises
// `st` and reads (and clears) that word, printing and remembering the code;
// it does nothing in release builds or while `st` is being captured.
// debug_take returns and clears the remembered code (0: none).
bool debug_build();
cudaError_t debug_check(cudaStream_t st, const char* what);
unsigned debug_take();

}  // namespace ptg
