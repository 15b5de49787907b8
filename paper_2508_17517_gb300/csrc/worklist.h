// One persistent launch per lockstep FGMRES iteration of many separate
// problems (grids of uneven size): the iteration's operations of every
// problem -- scale v_j, the V-cycle, w = A z_j, the Gram-Schmidt dots and
// update -- form a device work list of tiles that the blocks of one kernel
// take in order (worklist.cu).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "dev_util.cuh"
#include "handle.h"

namespace airg {

struct WorkList;   // worklist.cu

// Per-problem device pointers of the FGMRES state that the iteration reads
// and writes: Hessenberg column and <w,w> (h1, m + 2 entries), ||w||^2 after
// the update (nrm), the active flag.
struct WlProblem {
    Hierarchy* H;
    double* h1;
    double* nrm;
    const int* active;
};

// Whether every hierarchy's solve layout is one the work list implements:
// F-point smoothing with the matrix-free polynomial, FP64 or FP32 V-cycle
// (FP32 restrictor values, not bfloat16), no opt-in persistent or staged
// kernels, at most 8 warps per slice.
bool worklist_supported(const std::vector<Hierarchy*>& hs);

// Work list of iteration j (basis vectors v_0..v_j) for all problems.
std::shared_ptr<WorkList> build_worklist(const std::vector<WlProblem>& probs, int j, cudaStream_t st);

// Algorithmic bytes of problem `pr`'s operations in iteration j (stored
// entries and each vector read or written once, as the per-operator
// kernels count them), whichever form runs them.
long long iteration_bytes(const WlProblem& pr, int j);

// Clears the list's counters and launches its kernel on `st` (capturable).
void launch_worklist(WorkList& wl, cudaStream_t st);

// True (and clears the flag) if a wait of a launch of this list gave up.
bool worklist_timed_out(WorkList& wl, cudaStream_t st);

// Tiles and operations of the list (for reporting).
long long worklist_tiles(const WorkList& wl);
long long worklist_ops(const WorkList& wl);

}  // namespace airg
