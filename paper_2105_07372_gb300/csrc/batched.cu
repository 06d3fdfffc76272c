// Batched runs of Algorithm Synch-EM as one persistent kernel (config 4; the batching has no
// counterpart in the paper, which treats one problem at a time).
//
// One CTA per SM, launched cooperatively so that every CTA is resident.  Each iteration has two
// phases separated by a grid barrier:
//   sweep     items (instance i, CTA slot g < slots_i) taken from a global counter; a CTA runs
//             instance i's sweep body (Eq. weights_2d_em and Eq. coefficients_update over the
//             images of slot g) exactly as a launch of that sweep with grid slots_i would, and
//             leaves the slot's FP64 partials in the instance's workspace
//   finalize  items = instances: the column reduction in the fixed order of k_reduce_cols and the
//             update of k_finalize (a_{t+1}, rho_{t+1}, log-likelihood, step, stopping rule)
// so the arithmetic is that of the instance's own launches of the same sweep with grid slots_i (bit
// for bit where the lean sweep runs; the any-window warp sweep hands images out to its warps as they
// become free, so its FP32 sums vary in order from run to run).  Instances that have
// stopped (tolerance or their own iteration count) skip their items.  The grid barrier's wait is
// bounded: a CTA that gives up writes MRA_ETIMEOUT to the run's status word and leaves, and the
// others then give up at their next barrier.
#include "batched.cuh"
#include "sweep5_impl.cuh"
#include "sweep_impl.cuh"

namespace mra {

// Grid-wide barrier (arrival counter and generation in global memory); false if the wait ran out.
// The fences make every CTA's writes before the barrier visible to every CTA after it.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned long long limit_ns, int* status,
                             bool arrive = true) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    if (arrive && atomicAdd(bar, 1u) == nblocks - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (*vgen == gen) {
        if (globaltimer_ns() - t0 > limit_ns) {
          atomicExch(status, (int)MRA_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <int QV>
__device__ __forceinline__ void batched_sweep(const BatchedInst& I, int g) {
  const SweepV2Args& a = I.sa;
  switch (I.body) {
#define MRA_B5(MR)                                                   \
  case 2 * (MR - 1): sweep_v5_body<QV, MR, 20>(a, g, I.slots); break; \
  case 2 * (MR - 1) + 1: sweep_v5_body<QV, MR, 40>(a, g, I.slots); break;
    MRA_B5(1) MRA_B5(2) MRA_B5(3) MRA_B5(4) MRA_B5(5) MRA_B5(6) MRA_B5(7)
#undef MRA_B5
#define MRA_B2(MR) \
  case 16 + MR - 1: sweep_v2_body<QV, MR, 1, 0>(a, g, I.slots); break;
    MRA_B2(1) MRA_B2(2) MRA_B2(3) MRA_B2(4) MRA_B2(5) MRA_B2(6) MRA_B2(7)
#undef MRA_B2
    default: break;
  }
}

template <int QV>
__global__ void __launch_bounds__(kBatchedThreads, 1) k_em_batched(const BatchedArgs a) {
  __shared__ int s_item;
  const int tid = threadIdx.x, warp = tid >> 5, nw = kBatchedThreads / 32;
  const unsigned nblocks = gridDim.x;
  for (int t = 0; t < a.iters; ++t) {
    // ---- sweep items
    for (;;) {
      if (tid == 0) s_item = (int)atomicAdd(&a.counters[2 * t], 1u);
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= a.items) break;
      int lo = 0, hi = a.n - 1;  // the instance of this item: the last one starting at or before it
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.inst[mid].first_item <= item) lo = mid;
        else hi = mid - 1;
      }
      const BatchedInst& I = a.inst[lo];
      batched_sweep<QV>(I, item - I.first_item);
      __syncthreads();  // the next item reuses this CTA's shared memory
    }
    if (!grid_barrier(a.barrier, nblocks, a.limit_ns, a.status)) return;
    // ---- finalize items
    for (;;) {
      if (tid == 0) s_item = (int)atomicAdd(&a.counters[2 * t + 1], 1u);
      __syncthreads();
      const int i = s_item;
      __syncthreads();
      if (i >= a.n) break;
      const BatchedInst& I = a.inst[i];
      if (!__ldcg(&I.ctrl->done)) {
        for (int col = warp; col < I.cols; col += nw) reduce_cols_warp(I.part, I.slots, col, I.tot);
        __syncthreads();
        update_body(I.ua);
      }
      __syncthreads();
    }
    if (!grid_barrier(a.barrier, nblocks, a.limit_ns, a.status)) return;
  }
}

__global__ void k_selftest_grid_barrier(unsigned* bar, int* status, unsigned long long limit_ns) {
  grid_barrier(bar, gridDim.x, limit_ns, status, blockIdx.x != 0);
}

int launch_em_batched(const BatchedArgs& a, int grid, int smem, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_em_batched<2>);
  if (raise_smem_limit(fn, smem) != MRA_OK) return MRA_ECUDA;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBatchedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_em_batched<2>, a) == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

int batched_static_smem() {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k_em_batched<2>)) != cudaSuccess) return 64 * 1024;
  return (int)fa.sharedSizeBytes;
}

int launch_selftest_grid_barrier(int grid, unsigned* barrier, int* status, unsigned long long limit_ns,
                                 cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_selftest_grid_barrier, barrier, status, limit_ns) == cudaSuccess ? MRA_OK
                                                                                                         : MRA_ECUDA;
}

}  // namespace mra
