// Batched runs as one persistent kernel: the types shared by the host code (em.cu) and the kernel
// (batched.cu).
#pragma once
#include "common.cuh"
#include "update_impl.cuh"

namespace mra {

constexpr int kBatchedThreads = 512;

// One instance of a persistent batched run: its sweep (one of the bodies below, run once per CTA
// slot g < slots with the arguments' partial-sum stride sa.G = slots), its column reduction and
// its update, all on its own EM workspace.
struct BatchedInst {
  SweepV2Args sa;
  UpdateArgs ua;
  int body;        // sweep body id (batched_body_id), fixed at compile time in the kernel
  int slots;       // CTA slots of the sweep
  int first_item;  // index of the instance's first sweep item
  int cols;        // reduced columns (2M + Lw + 2)
  double* part;    // [cols][slots] per-slot partials
  double* tot;     // [cols + 8] totals
  Ctrl* ctrl;
};

struct BatchedArgs {
  const BatchedInst* inst;
  int n;                        // instances
  int items;                    // sweep items (sum of slots)
  int iters;                    // the largest max_iters (instances that stop earlier skip their items)
  unsigned* counters;           // [2 iters] item counters, zero at launch
  unsigned* barrier;            // [2] grid barrier: arrivals, generation (zero at launch)
  int* status;                  // MRA_OK; MRA_ETIMEOUT once a grid barrier wait ran out
  unsigned long long limit_ns;  // bound of every grid barrier wait
};

// Sweep bodies built into the persistent kernel (rows of 16 coefficients): the lean warp sweep for
// 1 <= MR <= 7 rows per quad and unit pitch 20 or 40 (ids 0..13: 2 (MR - 1) + (nup == 40)), and
// the warp sweep's any-window instance for 1 <= MR <= 7 (ids 16 + MR - 1).  -1: not built.
inline int batched_body_id(int Q, bool lean, int MR, int nup, int lwc) {
  if (Q != 16 || MR < 1 || MR > 7) return -1;
  if (lean) return (nup == 20 || nup == 40) ? 2 * (MR - 1) + (nup == 40 ? 1 : 0) : -1;
  return lwc == 0 ? 16 + MR - 1 : -1;
}

// Cooperative launch of the persistent kernel on `grid` CTAs (at most one per SM) with `smem`
// bytes of dynamic shared memory; raises the kernel's shared-memory limit first.
int launch_em_batched(const BatchedArgs& a, int grid, int smem, cudaStream_t s);
// Static shared memory of the persistent kernel (the sweep bodies' own arrays), which its dynamic
// shared memory must leave room for.
int batched_static_smem();
// Self-test of the grid barrier (no counterpart in the paper): `grid` CTAs meet at one barrier that
// CTA 0 never reaches; the others give up after limit_ns and write MRA_ETIMEOUT to *status.
int launch_selftest_grid_barrier(int grid, unsigned* barrier, int* status, unsigned long long limit_ns,
                                 cudaStream_t s);

}  // namespace mra
