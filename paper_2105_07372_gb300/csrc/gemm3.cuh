// C = A B^T on the tcgen05 tensor cores with FP32 operands split into three BF16 pieces
// (v = h + m + l, each the BF16 rounding of what the previous pieces leave): the six products
// hh, hm, mh, hl, lh, mm (fast mode: hh, hm, mh) accumulate in FP32 in tensor memory, so the
// result carries about FP32 precision (the products dropped are below 2^-24 of |a b|).
//
//   A  FP32 [rows][K], row stride lda (4-byte aligned rows are enough): converted to the three
//      pieces by the CTA's producer warps, 128 rows x 32 columns per pipeline stage
//   B  packed once by k_gemm3_pack: for every 256-column tile nt and 32-wide K block kb the three
//      pieces of B^T's [256][32] block in the K-major core-matrix layout of tc::op_offset,
//      contiguous (48 KB), so that one bulk copy fills a stage
//
// Roles per CTA (448 threads): warps 0-7 produce A, warp 8 copies B, warp 9 issues the MMAs, warps
// 10-13 run the epilogue (tile row 32 (w % 4) + lane = tensor-memory lane).  Stages are released by
// tcgen05.commit; every wait is bounded and reports MRA_ETIMEOUT through the status word.
// Output tiles are taken in groups that cover every column tile of consecutive row tiles, so
// that CTAs working at the same time share A rows and B tiles through L2.
#pragma once
#include <cuda_bf16.h>

#include "tc.cuh"

namespace mra {

constexpr int kG3Rows = 128, kG3Cols = 256, kG3KB = 32, kG3Stages = 3, kG3Threads = 448;
constexpr int kG3ATile = kG3Rows * kG3KB * 2;  // bytes of one A piece per stage
constexpr int kG3BTile = kG3Cols * kG3KB * 2;  // bytes of one B piece per stage
constexpr int kG3Stage = 3 * kG3ATile + 3 * kG3BTile;
constexpr int kG3Smem = 1024 + kG3Stages * kG3Stage;

struct Gemm3Args {
  const float* A;
  long long lda;
  int rows, K;
  const void* Bp;  // packed B: [NT][KB][3][brows x 32 BF16]
  int NT, KB, cols;
  int brows;       // rows of a packed B tile (a multiple of 16, <= 256; the MMAs' N)
  int nprod;       // 6 (accurate) or 3 (fast)
  float* C;        // store epilogue: C [rows][cols], row stride ldc
  long long ldc;
  // nearest-reference epilogue: out[i] = phi[argmin_j (rn[j] - 2 (A B^T)_ij)], j < cols, j != i
  const float* rn;
  const int* phi;
  int* out;
  int* status;
};

__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Pack B^T: element (j, k) of the [cols][K] matrix read as Bt(j, k) = src[j * sj + k * sk], into tiles of
// brows columns (the last one zero padded).
static __global__ void k_gemm3_pack(const float* src, long long sj, long long sk, int cols, int K, int NT, int KB,
                                    int brows, unsigned char* out) {
  const long long n = (long long)NT * brows * KB * kG3KB;
  const int ptile = brows * kG3KB * 2;  // bytes of one piece of a tile
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    // idx runs over (k, j) with j fastest: consecutive threads read consecutive columns
    const long long kk = idx / (NT * brows);
    const int jj = (int)(idx - kk * (NT * brows));
    const int k = (int)kk;
    float v = 0.f;
    if (jj < cols && k < K) v = src[jj * sj + k * sk];
    __nv_bfloat16 h, m, l;
    split3(v, h, m, l);
    const int nt = jj / brows, r = jj % brows, kb = k / kG3KB, c = k % kG3KB;
    unsigned char* chunk = out + ((size_t)nt * KB + kb) * (3 * ptile);
    const int off = tc::op_offset(r, c, kG3KB);
    *reinterpret_cast<__nv_bfloat16*>(chunk + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(chunk + ptile + off) = m;
    *reinterpret_cast<__nv_bfloat16*>(chunk + 2 * ptile + off) = l;
  }
}

// EPI 0: store C, accumulated over K segments of kG3Seg blocks; EPI 1: nearest reference (cols <= 256,
// one column tile, one segment).  The tensor core's FP32 accumulation loses precision over long sums
// (16,641-term projections cancel to 1/20 of their absolute sum), so the store epilogue restarts the
// accumulator every kG3Seg blocks and adds the partials in FP32 on the CUDA cores in a fixed order;
// two accumulators alternate so that the MMAs never wait for the addition.
constexpr int kG3Seg = 32;
template <int EPI>
__global__ void __launch_bounds__(kG3Threads, 1) k_gemm3(const Gemm3Args a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* full_a = reinterpret_cast<uint64_t*>(smem);        // [stages], 256 producer arrivals
  uint64_t* full_b = full_a + kG3Stages;                       // [stages], bulk-copy bytes
  uint64_t* empty = full_b + kG3Stages;                        // [stages], MMA commit
  uint64_t* acc_full = empty + kG3Stages;                      // [2] MMA commit after a segment
  uint64_t* acc_empty = acc_full + 2;                          // [2] 128 epilogue arrivals
  uint32_t* tbase_s = reinterpret_cast<uint32_t*>(acc_empty + 2);
  unsigned char* stages = smem + 1024;
  if (tid == 0) {
    for (int s = 0; s < kG3Stages; ++s) {
      mbar_init(&full_a[s], 2 * kG3Rows);
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kG3Rows);
    }
    fence_barrier_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tbase_s, 2u * kG3Cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tbase_s;
  const int MT = (a.rows + kG3Rows - 1) / kG3Rows;
  const int items = MT * a.NT;
  const int seg = EPI == 0 ? kG3Seg : a.KB;  // k blocks per accumulator segment
  const int nseg = (a.KB + seg - 1) / seg;
  // item it = row tile it / NT, column tile it % NT: the CTAs working at one time cover every
  // column tile of about gridDim / NT consecutive row tiles
  bool failed = false;
  auto wait = [&](uint64_t* b, uint32_t par) {
    if (failed) return false;
    if (!mbar_wait_bounded(b, par)) {
      failed = true;
      atomicExch(a.status, (int)MRA_ETIMEOUT);
      return false;
    }
    return true;
  };
  if (warp < 8) {
    // ---- A producers: lane l of warp w holds rows 16 w + 8 i + l / 4 (i = 0, 1), columns 8 (l % 4) .. + 7
    // of a k block; the next block's values are loaded (into registers) before this one is converted
    const int c0 = 8 * (lane & 3);
    const bool vec = (a.lda % 4) == 0 && (reinterpret_cast<uintptr_t>(a.A) % 16) == 0;
    auto load_blk = [&](int row0, int kb, float (&v)[2][8]) {
      const int k0 = kb * kG3KB + c0;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int gr = row0 + 16 * warp + 8 * i + (lane >> 2);
        const float* src = a.A + (long long)gr * a.lda + k0;
        if (vec && gr < a.rows && k0 + 8 <= a.K) {
          const float4 u = __ldg(reinterpret_cast<const float4*>(src)), w = __ldg(reinterpret_cast<const float4*>(src) + 1);
          v[i][0] = u.x, v[i][1] = u.y, v[i][2] = u.z, v[i][3] = u.w, v[i][4] = w.x, v[i][5] = w.y, v[i][6] = w.z, v[i][7] = w.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[i][e] = (gr < a.rows && k0 + e < a.K) ? __ldg(src + e) : 0.f;
        }
      }
    };
    int kiter = 0;
    for (int it = blockIdx.x; it < items && !failed; it += gridDim.x) {
      const int row0 = (it / a.NT) * kG3Rows;
      float cur[2][8], nxt[2][8];
      load_blk(row0, 0, cur);
      for (int kb = 0; kb < a.KB; ++kb, ++kiter) {
        if (kb + 1 < a.KB) load_blk(row0, kb + 1, nxt);
        const int s = kiter % kG3Stages;
        if (!wait(&empty[s], (uint32_t)(((kiter / kG3Stages) & 1) ^ 1))) break;
        unsigned char* st = stages + (size_t)s * kG3Stage;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int r = 16 * warp + 8 * i + (lane >> 2);
          __align__(16) __nv_bfloat16 ph[8], pm[8], pl[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) split3(cur[i][e], ph[e], pm[e], pl[e]);
          const int off = tc::op_offset(r, c0, kG3KB);
          *reinterpret_cast<uint4*>(st + off) = *reinterpret_cast<const uint4*>(ph);
          *reinterpret_cast<uint4*>(st + kG3ATile + off) = *reinterpret_cast<const uint4*>(pm);
          *reinterpret_cast<uint4*>(st + 2 * kG3ATile + off) = *reinterpret_cast<const uint4*>(pl);
        }
        tc::fence_proxy_async();
        mbar_arrive(&full_a[s]);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int e = 0; e < 8; ++e) cur[i][e] = nxt[i][e];
      }
    }
  } else if (warp == 8) {
    // ---- B producer: one bulk copy of the three pieces per stage
    if (lane == 0) {
      int kiter = 0;
      for (int it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        const int nt = it % a.NT;
        const uint32_t ptile = (uint32_t)a.brows * kG3KB * 2;
        const unsigned char* src = static_cast<const unsigned char*>(a.Bp) + (size_t)nt * a.KB * (3 * ptile);
        for (int kb = 0; kb < a.KB; ++kb, ++kiter) {
          const int s = kiter % kG3Stages;
          if (!wait(&empty[s], (uint32_t)(((kiter / kG3Stages) & 1) ^ 1))) break;
          unsigned char* st = stages + (size_t)s * kG3Stage + 3 * kG3ATile;
          const uint32_t bytes = (a.nprod > 3 ? 3 : 2) * ptile;  // the fast mode reads no l piece
          mbar_arrive_expect_tx(&full_b[s], bytes);
          bulk_g2s(st, src + (size_t)kb * (3 * ptile), bytes, &full_b[s]);
        }
      }
      if (failed) {  // copies this warp issued land before the CTA exits (each wait bounded)
        for (int u = max(0, kiter - kG3Stages); u < kiter; ++u)
          mbar_wait_bounded(&full_b[u % kG3Stages], (uint32_t)((u / kG3Stages) & 1));
      }
    }
  } else if (warp == 9) {
    // ---- MMA issuer: accumulator sc & 1 for the sc-th segment of this CTA
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kG3Rows, a.brows);
      const uint32_t ptile = (uint32_t)a.brows * kG3KB * 2;
      constexpr uint32_t SBO = (kG3KB / 8) * 128;
      int kiter = 0, sc = 0;
      for (int it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        for (int g = 0; g < nseg && !failed; ++g, ++sc) {
          const int b = sc & 1;
          if (!wait(&acc_empty[b], (uint32_t)(((sc >> 1) & 1) ^ 1))) break;
          tc::fence_after_sync();
          const uint32_t dacc = tbase + (uint32_t)(b * kG3Cols);
          const int kb1 = min(a.KB, (g + 1) * seg);
          for (int kb = g * seg; kb < kb1; ++kb, ++kiter) {
            const int s = kiter % kG3Stages;
            const uint32_t par = (uint32_t)((kiter / kG3Stages) & 1);
            if (!wait(&full_a[s], par) || !wait(&full_b[s], par)) break;
            tc::fence_after_sync();
            const uint32_t sa = smem_addr(stages + (size_t)s * kG3Stage);
            const uint32_t sb = sa + 3 * kG3ATile;
#pragma unroll
            for (int ks = 0; ks < kG3KB / 16; ++ks) {
              const uint32_t ko = ks * 256;
              const uint64_t ah = tc::smem_desc(sa + ko, 128, SBO), am = tc::smem_desc(sa + kG3ATile + ko, 128, SBO),
                             al = tc::smem_desc(sa + 2 * kG3ATile + ko, 128, SBO);
              const uint64_t bh = tc::smem_desc(sb + ko, 128, SBO), bm = tc::smem_desc(sb + ptile + ko, 128, SBO),
                             bl = tc::smem_desc(sb + 2 * ptile + ko, 128, SBO);
              const uint32_t first = (kb == g * seg && ks == 0) ? 0u : 1u;
              tc::mma_f16(dacc, ah, bh, idesc, first);
              tc::mma_f16(dacc, ah, bm, idesc, 1u);
              tc::mma_f16(dacc, am, bh, idesc, 1u);
              if (a.nprod > 3) {
                tc::mma_f16(dacc, ah, bl, idesc, 1u);
                tc::mma_f16(dacc, al, bh, idesc, 1u);
                tc::mma_f16(dacc, am, bm, idesc, 1u);
              }
            }
            tc::mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
          }
          if (failed) break;
          tc::mma_commit(&acc_full[b]);
        }
      }
    }
  } else {
    // ---- epilogue warps 10..13: tile row = 32 (warp % 4) + lane = tensor-memory lane
    const int qtr = warp & 3, row = 32 * qtr + lane;
    int sc = 0;
    for (int it = blockIdx.x; it < items && !failed; it += gridDim.x) {
      const int mt = it / a.NT, nt = it % a.NT;
      const int gr = mt * kG3Rows + row;
      float best = INFINITY;
      int bj = 0;
      for (int g = 0; g < nseg; ++g, ++sc) {
        const int b = sc & 1;
        if (!wait(&acc_full[b], (uint32_t)((sc >> 1) & 1))) break;
        tc::fence_after_sync();
        const uint32_t trow = tbase + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(b * kG3Cols);
        if (EPI == 0) {
          const int col0 = nt * a.brows;
          for (int c = 0; c < a.brows; c += 16) {
            float v[16];
            tc::tmem_ld16(trow + (uint32_t)c, v);
            if (gr < a.rows) {
              float* dst = a.C + (long long)gr * a.ldc + col0 + c;
              if (col0 + c + 16 <= a.cols && (a.ldc & 3) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                  if (g > 0) {  // this thread wrote the earlier segments' sum itself
                    const float4 p = reinterpret_cast<float4*>(dst)[q];
                    o.x += p.x, o.y += p.y, o.z += p.z, o.w += p.w;
                  }
                  reinterpret_cast<float4*>(dst)[q] = o;
                }
              } else {
                for (int q = 0; q < 16; ++q)
                  if (col0 + c + q < a.cols) dst[q] = g > 0 ? dst[q] + v[q] : v[q];
              }
            }
          }
        } else {
          for (int c = 0; c < a.brows; c += 16) {
            float v[16];
            tc::tmem_ld16(trow + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int jc = c + q;
              if (jc < a.cols && jc != gr) {
                const float dist = fmaf(-2.f, v[q], a.rn[jc]);
                if (dist < best) best = dist, bj = jc;
              }
            }
          }
        }
        tc::fence_before_sync();
        mbar_arrive(&acc_empty[b]);
      }
      if (EPI == 1 && !failed && gr < a.rows) a.out[gr] = a.phi[bj];
    }
  }
  // every role leaves its loop; drain before the tensor memory is freed
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 2u * kG3Cols);
}

}  // namespace mra
