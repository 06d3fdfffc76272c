// Split EM sweep for wide windows (Eq. weights_2d_em, Eq. coefficients_update) with the window
// transform on the tensor cores.
//
//   k_tc_corr   warp per image (quad layout of the warp sweeps, packed FP32 FMAs): the aligned
//               correlations c_jk = e^{-i k theta_hat_j} sum_q conj(y_jkq) x_kq to a buffer [N][K+1]
//   k_tc_trans  tiles of 128 images, thread t = image t = tensor-memory lane t:
//                 pass 1  S_jl = Re sum_k c_jk e^{-i k theta_l} for every window rotation as one
//                         tcgen05 MMA per 16 columns of K: A = [c.re, c.im] rows in FP16 (hi + lo
//                         split after a per-image power-of-two scale), B = [cos, sin] of the window
//                         rotations in FP16, FP32 accumulation in tensor memory (windows of more than
//                         512 rotations in passes of 512 columns, the earlier ones computed again for
//                         the cut).  Each thread reads its
//                         row, finds the peak l* and the distance D beyond which every log-weight is
//                         more than 40 below it, widened by twice a bound on pass 1's rounding
//                         (FP16 twiddles: 2^-12 per entry, times sum_k |c.re| + |c.im|)
//                 pass 2  as in the other sweeps, exact FP32 differences from the peak from c rotated to
//                         the peak and the FP64-built (cos t - 1, -sin t) table, over d <= D: the
//                         maximum and normaliser in one pass, the weights and the back transform
//                         W_k = e^{i k theta_l*} (1 + sum_d ...) in a second, W_t[l] in 2^-40
//                         fixed point (integer shared-memory atomics, order-independent)
//   k_tc_accum  warp per image: num_kq += W_jk y_jkq into per-lane FP32 registers
//
// y is read twice (correlation and accumulation); the transform works on 16 + 16 bytes per image
// and rotation.  Partial sums go to the per-CTA FP64 columns of the EM workspace as in the fused
// sweeps: num (k_tc_accum), W_t and the log-likelihood (k_tc_trans), sum ||y||^2 (k_tc_corr).
#pragma once
#include "tc.cuh"

namespace mra {


__device__ __forceinline__ int tc_mod(int a, int L, float invL) {
  int m = a - __float2int_rz((float)a * invL) * L;
  if (m < 0) m += L;
  if (m >= L) m -= L;
  return m;
}

// ---------------------------------------------------------------- correlation
template <int QV, int MR>
__global__ void __launch_bounds__(kTcStreamThreads, 1) k_tc_corr(const SplitArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = kTcStreamThreads, row4 = QV * 4;
  constexpr unsigned FULL = 0xffffffffu;
  if (a.ctrl->done) return;
  const bool want_ysq = (a.ctrl->iter == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = a.nwarps, r = lane >> 2, j = lane & 3;
  const int Kp1 = a.Kp1, L = a.L, M = a.M;
  const float invL = 1.0f / (float)L;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* ring = smem + a.off_ring;
  const float4* xs4 = reinterpret_cast<const float4*>(smem + a.off_x);
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);
  {
    float4* x4w = reinterpret_cast<float4*>(smem + a.off_x);
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
    for (int i = tid; i < M / 2; i += NT) {
      const float4 v = xg[i];
      x4w[i] = v;
    }
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    if (tid < 2 * nwarps) mbar_init(&bar[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();
  const int gw = blockIdx.x * nwarps + warp, GW = gridDim.x * nwarps;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  unsigned char* const wring = ring + (size_t)warp * 2 * a.slot_bytes;
  uint64_t* mybar = bar + 2 * warp;
  auto issue = [&](int im, int st) {
    if (im >= a.N) return;
    mbar_arrive_expect_tx(&mybar[st], img_bytes);
    bulk_g2s(wring + (size_t)st * a.slot_bytes, a.y + (size_t)im * M, img_bytes, &mybar[st]);
  };
  auto load_shift = [&](int im) -> int {
    if (!a.shift || im >= a.N) return 0;
    int s = a.shift[im];
    if (s < 0 || s >= L) {
      s %= L;
      if (s < 0) s += L;
    }
    return s;
  };
  double ysq_acc = 0.0;
  if (warp < nwarps && lane == 0) {
    issue(gw, 0);
    issue(gw + GW, 1);
  }
  int sj_next = warp < nwarps ? load_shift(gw) : 0;
  for (int it = 0; warp < nwarps && gw + it * GW < a.N; ++it) {
    const int st = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const int img = gw + it * GW;
    const int sj = sj_next;
    sj_next = load_shift(img + GW);
    const bool ok = mbar_wait_bounded(&mybar[st], parity);
    if (!__all_sync(FULL, ok)) {
      if (lane == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        mbar_wait_bounded(&mybar[st], parity);
        if (img + GW < a.N) mbar_wait_bounded(&mybar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
      }
      break;
    }
    const float4* y4 = reinterpret_cast<const float4*>(wring + (size_t)st * a.slot_bytes);
    float2 sq = make_float2(0.f, 0.f);
    int ph = tc_mod(r * sj, L, invL);
    const int pst = tc_mod(8 * sj, L, invL);
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int k = r + 8 * m;
      float2 P = make_float2(0.f, 0.f), Qv = make_float2(0.f, 0.f);
      if (m < MR - 1 || k < Kp1) {
#pragma unroll
        for (int u = 0; u < QV; ++u) {
          const int pidx = k * row4 + j + 4 * u;
          const float4 yv = y4[pidx], xv = xs4[pidx];
          const float2 y01 = make_float2(yv.x, yv.y), y23 = make_float2(yv.z, yv.w);
          P = __ffma2_rn(y01, make_float2(xv.x, xv.y), P);
          P = __ffma2_rn(y23, make_float2(xv.z, xv.w), P);
          Qv = __ffma2_rn(y01, make_float2(xv.y, xv.x), Qv);  // (y.re x.im, y.im x.re): Im c is their difference
          Qv = __ffma2_rn(y23, make_float2(xv.w, xv.z), Qv);
          if (want_ysq) {
            sq = __ffma2_rn(y01, y01, sq);
            sq = __ffma2_rn(y23, y23, sq);
          }
        }
      }
      float cr = P.x + P.y, ci = Qv.x - Qv.y;
      cr += __shfl_xor_sync(FULL, cr, 1);
      ci += __shfl_xor_sync(FULL, ci, 1);
      cr += __shfl_xor_sync(FULL, cr, 2);
      ci += __shfl_xor_sync(FULL, ci, 2);
      float2 cv = make_float2(cr, ci);
      if (a.shift) cv = cmul(cv, tfs[ph]);  // c_k e^{-i k theta_hat_j}
      ph += pst;
      if (ph >= L) ph -= L;
      if (j == 0 && (m < MR - 1 || k < Kp1)) a.cbuf[(size_t)img * Kp1 + k] = cv;
    }
    if (want_ysq) {
      const float t = warp_sum(sq.x + sq.y);
      if (lane == 0) ysq_acc += (double)t;
    }
    __syncwarp();
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(img + 2 * GW, st);
    }
  }
  __shared__ double red[32];
  if (lane == 0) red[warp] = ysq_acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    a.part[(size_t)(2 * M + a.Lw + 1) * a.G + blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- transform (tensor cores)
// 512 threads per tile of 128 images.  Pass 1's row of image i is tensor-memory lane i: warp w reads
// the lanes of quarter w % 4 over the column block w / 4, the four blocks' maxima are combined in
// shared memory.  Pass 2 and the back transform run on a warp per image (lanes over distances for
// the values, over rows for the back transform), the images of the tile handed out to the warps
// from a counter.
// KP: K+1 rounded up to a multiple of 4; the MMA's K is 2 KP rounded up to 16.
template <int KP>
__global__ void __launch_bounds__(kTcTransThreads, 1) k_tc_trans(const SplitArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int KA = (2 * KP + 15) / 16 * 16;
  constexpr int SBO = (KA / 8) * 128;  // bytes between 8-row groups of an operand
  constexpr int NT = kTcTransThreads;
  constexpr int TP = KP + 1;  // pitch of a distance's row in the shared table (odd: no bank conflicts)
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int s_next;  // the tile's next image for pass 2
  if (a.ctrl->done) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Kp1 = a.Kp1, L = a.L, Lw = a.Lw, NP = a.NP, M = a.M;
  const bool wrap = a.wrap != 0, dense = a.tw != nullptr;
  const float two_beta = a.two_beta;
  const float invL = 1.0f / (float)L;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tbase_s = reinterpret_cast<uint32_t*>(smem + 8);
  unsigned char* Bs = smem + a.k2_off_b;   // [NP][KA] FP16 operand layout
  unsigned char* Ah = smem + a.k2_off_ah;  // [128][KA]
  unsigned char* Al = smem + a.k2_off_al;
  float* lrs = reinterpret_cast<float*>(smem + a.k2_off_lr);                            // [Lw]
  float2* tfs = reinterpret_cast<float2*>(smem + a.k2_off_tf);                         // [L]
  unsigned long long* wts = reinterpret_cast<unsigned long long*>(smem + a.k2_off_wt);  // [Lw]
  float2* swb = reinterpret_cast<float2*>(smem + a.k2_off_ll);  // [NT / 32][32] back-transform terms
  float2* cst = reinterpret_cast<float2*>(smem + a.k2_off_cs);                         // [128][Kp1] c, then W
  float* ibest = reinterpret_cast<float*>(smem + a.k2_off_info);  // [4][128] block maxima
  int* ibl = reinterpret_cast<int*>(ibest + 4 * kTcTile);          // [4][128] their window indices
  int* iD = ibl + 4 * kTcTile;                                     // [4][128] block distances
  float* iscale = reinterpret_cast<float*>(iD + 4 * kTcTile);      // [128] A row scale
  float* ibound = iscale + kTcTile;                                // [128] pass-1 rounding bound
  double* lli = reinterpret_cast<double*>(ibest);                   // [128] log-likelihoods (pass 2)
  int* iDm = reinterpret_cast<int*>(ibest + 2 * kTcTile);           // [128] D of each image (pass 2)
  int* iord = iDm + kTcTile;                                       // [128] images by decreasing D
  // the distance-unit table's first k2_ndp distances, [d][TP] (rows k >= K+1 zero)
  float2* tds = a.k2_off_td ? reinterpret_cast<float2*>(smem + a.k2_off_td) : nullptr;
  {
    const uint4* bg = reinterpret_cast<const uint4*>(a.tcb);
    uint4* bw = reinterpret_cast<uint4*>(Bs);
    for (int i = tid; i < NP * KA / 8; i += NT) bw[i] = bg[i];
    for (int i = tid; i < Lw; i += NT) lrs[i] = a.logrho32[i], wts[i] = 0ull;
    for (int i = tid; i < L; i += NT) tfs[i] = a.tf32[i];
    if (tds)  // the first k2_ndp distances of every row (the ones near each image's peak)
      for (int i = tid; i < TP * a.k2_ndp; i += NT) {
        const int d = i / TP, k = i - d * TP;
        tds[i] = k < Kp1 ? a.td[k * a.nd + d] : make_float2(0.f, 0.f);
      }
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_barrier_init();
    }
  }
  const int ndp = tds ? a.k2_ndp : 0;
  if (warp == 0) {
    tc::tmem_alloc(tbase_s, (uint32_t)a.ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tbase_s;
  const int qtr = warp & 3, cblk = warp >> 2;
  const uint32_t trow = tbase + ((uint32_t)(qtr * 32) << 16);  // this warp's lanes
  const uint32_t ah_addr = smem_addr(Ah), al_addr = smem_addr(Al), b_addr = smem_addr(Bs);
  const int nd1 = a.nd - 1;
  double ll_acc = 0.0;
  uint32_t phase = 0;
  const int ntiles = (a.N + kTcTile - 1) / kTcTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int img0 = tile * kTcTile;
    const int nimg = min(kTcTile, a.N - img0);
    // ---- the tile's aligned correlations (one coalesced copy)
    for (int i = tid; i < nimg * Kp1; i += NT) cst[i] = a.cbuf[(size_t)img0 * Kp1 + i];
    __syncthreads();
    // ---- A rows (FP16 hi + lo of s c), threads 0..127: one image each
    if (tid < kTcTile) {
      const bool valid = tid < nimg;
      float mxabs = 0.f, sumabs = 0.f;
      for (int k = 0; k < Kp1; ++k) {
        const float2 v = valid ? cst[tid * Kp1 + k] : make_float2(0.f, 0.f);
        mxabs = fmaxf(mxabs, fmaxf(fabsf(v.x), fabsf(v.y)));
        sumabs += fabsf(v.x) + fabsf(v.y);
      }
      int ex = 0;
      frexpf(mxabs, &ex);
      const float scale = mxabs > 0.f ? ldexpf(1.f, 14 - ex) : 1.f;  // scale * |c| < 2^14
      iscale[tid] = scale;
      ibound[tid] = two_beta * sumabs * 2.5e-4f;  // FP16 twiddles and FP32 sums of pass 1
#pragma unroll
      for (int kc = 0; kc < KA / 8; ++kc) {
        __align__(16) __half hv[8], lv[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * kc + e;
          const float2 c0 = (valid && k < Kp1) ? cst[tid * Kp1 + k] : make_float2(0.f, 0.f);
          const float2 v = make_float2(c0.x * scale, c0.y * scale);
          const __half hx = __float2half_rn(v.x), hy = __float2half_rn(v.y);
          hv[2 * e] = hx;
          hv[2 * e + 1] = hy;
          lv[2 * e] = __float2half_rn(v.x - __half2float(hx));
          lv[2 * e + 1] = __float2half_rn(v.y - __half2float(hy));
        }
        const int off = tc::op_offset(tid, 8 * kc, KA);
        *reinterpret_cast<uint4*>(Ah + off) = *reinterpret_cast<const uint4*>(hv);
        *reinterpret_cast<uint4*>(Al + off) = *reinterpret_cast<const uint4*>(lv);
      }
      tc::fence_proxy_async();
    }
    tc::fence_before_sync();
    __syncthreads();
    // ---- pass 1 on the tensor cores: D[128][NP] = (A_hi + A_lo) B^T, in passes of at most 512 window
    // columns (the tensor memory of one CTA); a second pass's columns reuse the same tensor memory
    auto run_mma = [&](int base) -> bool {  // the caller has fenced and synchronised the previous reads
      if (tid == 0) {
        tc::fence_after_sync();
        const int hi = min(NP, base + 512);
        for (int n0 = base; n0 < hi; n0 += 256) {
          const int nc = hi - n0 < 256 ? hi - n0 : 256;
          const uint32_t idesc = tc::idesc_f16(kTcTile, nc);
#pragma unroll
          for (int ks = 0; ks < KA / 16; ++ks) {
            const uint64_t bd = tc::smem_desc(b_addr + (uint32_t)((n0 / 8) * SBO + ks * 256), 128, SBO);
            tc::mma_f16(tbase + (uint32_t)(n0 - base), tc::smem_desc(ah_addr + ks * 256, 128, SBO), bd, idesc,
                        ks > 0 ? 1u : 0u);
            tc::mma_f16(tbase + (uint32_t)(n0 - base), tc::smem_desc(al_addr + ks * 256, 128, SBO), bd, idesc, 1u);
          }
        }
        tc::mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) {
          atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
          mbar_wait_bounded(bar, phase ^ 1u);  // let the MMAs in flight finish before the memory is freed
        }
        return false;
      }
      tc::fence_after_sync();
      return true;
    };
    // this warp's column block of a pass: 4 blocks of 16-column groups over the pass's columns
    auto block = [&](int base, int& lo, int& hi) {
      const int pc = min(512, NP - base), nq = ((pc + 3) / 4 + 15) / 16 * 16;
      lo = base + cblk * nq;
      hi = min(base + pc, lo + nq);
    };
    const int npass = (NP + 511) / 512;
    bool failed = false;
    // ---- the peak: each warp over its column blocks of its 32 lanes (images 32 qtr + lane)
    {
      const int row = qtr * 32 + lane;
      const float kap = two_beta / iscale[row];
      float best = -INFINITY;
      int bl = 0x7fffffff;
      for (int ps = 0; ps < npass; ++ps) {
        if (ps > 0) {
          tc::fence_before_sync();
          __syncthreads();
        }
        if (!run_mma(512 * ps)) {
          failed = true;
          break;
        }
        int lo, hi;
        block(512 * ps, lo, hi);
        for (int c0 = lo; c0 < hi; c0 += 16) {
          float v[16];
          tc::tmem_ld16(trow + (uint32_t)(c0 - 512 * ps), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int l = c0 + i;
            if (l < Lw) {
              const float sv = fmaf(kap, v[i], lrs[l]);
              if (sv > best) best = sv, bl = l;
            }
          }
        }
      }
      if (!failed) {
        ibest[cblk * kTcTile + row] = best;
        ibl[cblk * kTcTile + row] = bl;
      }
    }
    if (failed) break;
    __syncthreads();
    if (tid < kTcTile) {  // combine the blocks in order (the first maximum wins)
      float best = ibest[tid];
      int bl = ibl[tid];
      for (int b = 1; b < 4; ++b)
        if (ibest[b * kTcTile + tid] > best) best = ibest[b * kTcTile + tid], bl = ibl[b * kTcTile + tid];
      if (bl >= Lw || best == -INFINITY) bl = 0;
      ibest[tid] = best;
      ibl[tid] = bl;
    }
    if (tid == 0) s_next = 0;
    __syncthreads();
    // ---- the distance D beyond which every value is more than 40 (plus twice the bound) below the peak;
    // the last pass is still in tensor memory, earlier passes are computed again
    {
      const int row = qtr * 32 + lane;
      const float kap = two_beta / iscale[row];
      const float thr = ibest[row] - 40.f - 2.f * ibound[row];
      const int bl = ibl[row];
      int D = 0;
      for (int k = 0; k < npass; ++k) {
        const int ps = npass - 1 - k;
        if (k > 0) {
          tc::fence_before_sync();
          __syncthreads();
          if (!run_mma(512 * ps)) {
            failed = true;
            break;
          }
        }
        int lo, hi;
        block(512 * ps, lo, hi);
        for (int c0 = lo; c0 < hi; c0 += 16) {
          float v[16];
          tc::tmem_ld16(trow + (uint32_t)(c0 - 512 * ps), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int l = c0 + i;
            if (l < Lw && fmaf(kap, v[i], lrs[l]) >= thr) {
              int dd = l > bl ? l - bl : bl - l;
              if (wrap && L - dd < dd) dd = L - dd;
              D = max(D, dd);
            }
          }
        }
      }
      if (!failed) {
        tc::fence_before_sync();  // tensor memory is rewritten by the next tile's MMAs after a barrier
        __syncthreads();          // every block has read ibest/ibl
        iD[cblk * kTcTile + row] = D;
      }
    }
    if (failed) break;
    __syncthreads();
    // images in order of decreasing D (ties by index), so that the broadest posteriors start first and
    // the rest fill in around them
    if (tid < nimg) iDm[tid] = max(max(iD[tid], iD[kTcTile + tid]), max(iD[2 * kTcTile + tid], iD[3 * kTcTile + tid]));
    __syncthreads();
    if (tid < nimg) {
      const int Di = iDm[tid];
      int rank = 0;
      for (int j = 0; j < nimg; ++j) {
        const int Dj = iDm[j];
        rank += (Dj > Di || (Dj == Di && j < tid)) ? 1 : 0;
      }
      iord[rank] = tid;
    }
    __syncthreads();
    // ---- pass 2 and the back transform: a warp per image (images handed out from the tile's counter,
    // so that an image with a broad posterior holds one warp, not the tile), lanes over the distances
    // d = c0 + lane of chunks of 32 for the values and over the rows k = lane, lane + 32 for the back
    // transform; the rotated c of the image replaces its c in cst
    for (;;) {
      int n_ = 0;
      if (lane == 0) n_ = atomicAdd(&s_next, 1);
      n_ = __shfl_sync(FULL, n_, 0);
      if (n_ >= nimg) break;
      const int i = iord[n_];
      const int img = img0 + i;
      const int p = ibl[i];
      const int D = iDm[i];
      int op = 0;
      if (!dense) {
        op = a.l0m + p;
        if (op >= L) op -= L;
      }
      float2* cqi = cst + i * Kp1;
      float Sp = 0.f;
      for (int k = lane; k < Kp1; k += 32) {
        const float2 f = dense ? a.tw[k * a.twp + p] : tfs[tc_mod(k * op, L, invL)];
        const float2 cq = cmul(cqi[k], f);
        cqi[k] = cq;
        Sp += cq.x;
      }
      Sp = warp_sum(Sp);
      __syncwarp();
      const float lrp = lrs[p];
      // S(l* + d) - S(l*) and S(l* - d) - S(l*) at this lane's distance (-inf where absent)
      auto values = [&](int d, float& sp, float& sm, int& la, int& lb) {
        const int dc = d <= D ? min(d, nd1) : 0;  // lanes past D read the shared table (their values are unused)
        float2 ab = make_float2(0.f, 0.f);
        if (dc < ndp) {
          const float2* t = tds + dc * TP;
#pragma unroll 4
          for (int k = 0; k < KP; ++k)
            if (k < Kp1) ab = __ffma2_rn(cqi[k], t[k], ab);
        } else {
          const float2* t = a.td + dc;
#pragma unroll 4
          for (int k = 0; k < KP; ++k)
            if (k < Kp1) ab = __ffma2_rn(cqi[k], t[(size_t)k * a.nd], ab);
        }
        la = p + d;
        lb = p - d;
        bool vp, vm;
        if (wrap) {
          if (la >= L) la -= L;
          if (lb < 0) lb += L;
          vp = true;
          vm = d > 0 && 2 * d != L;
        } else {
          vp = la < Lw;
          vm = d > 0 && lb >= 0;
        }
        vp = vp && d <= D;
        vm = vm && d <= D;
        sp = vp ? fmaf(two_beta, ab.x - ab.y, lrs[min(max(la, 0), Lw - 1)] - lrp) : -INFINITY;
        sm = vm ? fmaf(two_beta, ab.x + ab.y, lrs[min(max(lb, 0), Lw - 1)] - lrp) : -INFINITY;
      };
      // values relative to the peak (the peak's own is exactly 0, none exceeds twice pass 1's bound):
      // the normaliser sums their exponentials directly
      float z = 0.f;
      for (int c0 = 0; c0 <= D; c0 += 32) {
        float sp, sm;
        int la, lb;
        values(c0 + lane, sp, sm, la, lb);
        z += expf(sp) + expf(sm);
      }
      z = warp_sum(z);
      if (lane == 0) lli[i] = (double)(lrp + two_beta * Sp) + (double)logf(z);
      const float inv = 1.f / z;
      float* wo = a.w_out ? a.w_out + (size_t)img * Lw : nullptr;
      if (wo) {
        for (int l = lane; l < Lw; l += 32) wo[l] = 0.f;
        __syncwarp();
      }
      const int k0 = lane, k1 = lane + 32;
      float2 W0 = make_float2(0.f, 0.f), W1 = make_float2(0.f, 0.f);
      float2* sw = swb + warp * 32;
      for (int c0 = 0; c0 <= D; c0 += 32) {
        float sp, sm;
        int la, lb;
        const int d = c0 + lane;
        values(d, sp, sm, la, lb);
        const float wp = expf(sp) * inv, wm = expf(sm) * inv;
        if (sp > -INFINITY) {
          atomicAdd(&wts[la], (unsigned long long)__float2ull_rn(wp * 1099511627776.f));
          if (wo) wo[la] = wp;
        }
        if (sm > -INFINITY) {
          atomicAdd(&wts[lb], (unsigned long long)__float2ull_rn(wm * 1099511627776.f));
          if (wo) wo[lb] = wm;
        }
        // back transform around the peak: W_k e^{-i k theta_l*} = 1 + sum_{d>=1} [(w_{+d} + w_{-d}) (cos t - 1)
        //   + i (w_{-d} - w_{+d}) (-sin t)], the chunk's terms staged per warp
        sw[lane] = d >= 1 ? make_float2(wp + wm, wm - wp) : make_float2(0.f, 0.f);
        __syncwarp();
        const int n = min(32, D + 1 - c0);
        if (c0 + n <= ndp) {
          for (int e = 0; e < n; ++e) {
            const float2 s = sw[e];
            const float2* t = tds + (c0 + e) * TP;
            W0 = __ffma2_rn(s, t[min(k0, KP - 1)], W0);
            if (KP > 32) W1 = __ffma2_rn(s, t[min(k1, KP - 1)], W1);
          }
        } else {
          for (int e = 0; e < n; ++e) {
            const float2 s = sw[e];
            const int dc = min(c0 + e, nd1);
            if (dc < ndp) {
              const float2* t = tds + dc * TP;
              W0 = __ffma2_rn(s, t[min(k0, KP - 1)], W0);
              if (KP > 32) W1 = __ffma2_rn(s, t[min(k1, KP - 1)], W1);
            } else {
              if (k0 < Kp1) W0 = __ffma2_rn(s, a.td[(size_t)k0 * a.nd + dc], W0);
              if (KP > 32 && k1 < Kp1) W1 = __ffma2_rn(s, a.td[(size_t)k1 * a.nd + dc], W1);
            }
          }
        }
        __syncwarp();  // the next chunk rewrites the stage
      }
      // W_k = e^{+i k (theta_hat_j + theta_l*)} (1 + sum ...): rotated back by the peak and the shift
      int sj = 0;
      if (a.shift) {
        sj = a.shift[img] % L;
        if (sj < 0) sj += L;
      }
      int q = dense ? sj : sj + op;
      if (q >= L) q -= L;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = h ? k1 : k0;
        if (k < Kp1) {
          const float2 Wd = h ? W1 : W0;
          float2 w = make_float2(1.f + Wd.x, Wd.y);
          if (dense) w = cmul_conj_b(w, a.tw[k * a.twp + p]);
          w = cmul_conj_b(w, tfs[tc_mod(k * q, L, invL)]);
          cqi[k] = w;  // this lane's own rows (every lane has read the rotated c above)
        }
      }
    }
    __syncthreads();
    if (tid < nimg) ll_acc += lli[tid];  // a fixed image per thread: the order is the same every run
    for (int i = tid; i < nimg * Kp1; i += NT) a.wbuf[(size_t)img0 * Kp1 + i] = cst[i];
    __syncthreads();  // the next tile's copy rewrites the stage
  }
  // ---- teardown and the CTA's partial sums (fixed order)
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, (uint32_t)a.ncols);
  double* llr = reinterpret_cast<double*>(cst);  // [NT]: the stage is free after the last tile
  llr[tid] = ll_acc;
  __syncthreads();
  const int G = a.G, cta = blockIdx.x;
  for (int l = tid; l < Lw; l += NT)
    a.part[(size_t)(2 * M + l) * G + cta] = (double)wts[l] * (1.0 / 1099511627776.0);
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < NT; ++i) t += llr[i];
    a.part[(size_t)(2 * M + Lw) * G + cta] = t;
  }
}

// ---------------------------------------------------------------- accumulation
template <int QV, int MR>
__global__ void __launch_bounds__(kTcStreamThreads, 1) k_tc_accum(const SplitArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = kTcStreamThreads, row4 = QV * 4;
  if (a.ctrl->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = a.nwarps, r = lane >> 2, j = lane & 3;
  const int Kp1 = a.Kp1, M = a.M;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* ring = smem + a.off_ring;
  if (tid < 2 * nwarps) mbar_init(&bar[tid], 1);
  if (tid == 0) fence_barrier_init();
  __syncthreads();
  const int gw = blockIdx.x * nwarps + warp, GW = gridDim.x * nwarps;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  unsigned char* const wring = ring + (size_t)warp * 2 * a.slot_bytes;
  uint64_t* mybar = bar + 2 * warp;
  auto issue = [&](int im, int st) {
    if (im >= a.N) return;
    mbar_arrive_expect_tx(&mybar[st], img_bytes);
    bulk_g2s(wring + (size_t)st * a.slot_bytes, a.y + (size_t)im * M, img_bytes, &mybar[st]);
  };
  auto load_w = [&](int im, float2 (&w)[MR]) {
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int k = r + 8 * m;
      w[m] = (im < a.N && (m < MR - 1 || k < Kp1)) ? a.wbuf[(size_t)im * Kp1 + k] : make_float2(0.f, 0.f);
    }
  };
  float4 acc[MR][QV];
#pragma unroll
  for (int m = 0; m < MR; ++m)
#pragma unroll
    for (int u = 0; u < QV; ++u) acc[m][u] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp < nwarps && lane == 0) {
    issue(gw, 0);
    issue(gw + GW, 1);
  }
  float2 wn[MR];
  if (warp < nwarps) load_w(gw, wn);
  for (int it = 0; warp < nwarps && gw + it * GW < a.N; ++it) {
    const int st = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const int img = gw + it * GW;
    float2 W[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) W[m] = wn[m];
    load_w(img + GW, wn);  // in flight while this image is accumulated
    const bool ok = mbar_wait_bounded(&mybar[st], parity);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        mbar_wait_bounded(&mybar[st], parity);
        if (img + GW < a.N) mbar_wait_bounded(&mybar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
      }
      break;
    }
    const float4* y4 = reinterpret_cast<const float4*>(wring + (size_t)st * a.slot_bytes);
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int k = r + 8 * m;
      if (m < MR - 1 || k < Kp1) {
        const float2 w = W[m];
#pragma unroll
        for (int u = 0; u < QV; ++u) {
          const float4 yv = y4[k * row4 + j + 4 * u];
          float4& q = acc[m][u];
          q.x = fmaf(w.x, yv.x, q.x); q.x = fmaf(-w.y, yv.y, q.x);
          q.y = fmaf(w.x, yv.y, q.y); q.y = fmaf(w.y, yv.x, q.y);
          q.z = fmaf(w.x, yv.z, q.z); q.z = fmaf(-w.y, yv.w, q.z);
          q.w = fmaf(w.x, yv.w, q.w); q.w = fmaf(w.y, yv.z, q.w);
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(img + 2 * GW, st);
    }
  }
  __syncthreads();
  float4* red4 = reinterpret_cast<float4*>(ring);  // [NT/32][M/2]
  const int half = M / 2;
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int k = r + 8 * m;
    if (m < MR - 1 || k < Kp1) {
#pragma unroll
      for (int u = 0; u < QV; ++u) red4[(size_t)warp * half + k * row4 + j + 4 * u] = acc[m][u];
    }
  }
  __syncthreads();
  const float* redf = reinterpret_cast<const float*>(ring);
  for (int col = tid; col < 2 * M; col += NT) {
    float sum = 0.f;
    for (int w = 0; w < NT / 32; ++w) sum += redf[(size_t)w * 2 * M + col];
    a.part[(size_t)col * a.G + blockIdx.x] = (double)sum;
  }
}

}  // namespace mra

#define MRA_SWEEP_TC_STREAM_TABLE(QV)                                                   \
  namespace mra {                                                                       \
  SplitStreamFns sweep_tc_q##QV(int MR) {                                               \
    switch (MR) {                                                                       \
      case 1: return {k_tc_corr<QV, 1>, k_tc_accum<QV, 1>};                             \
      case 2: return {k_tc_corr<QV, 2>, k_tc_accum<QV, 2>};                             \
      case 3: return {k_tc_corr<QV, 3>, k_tc_accum<QV, 3>};                             \
      case 4: return {k_tc_corr<QV, 4>, k_tc_accum<QV, 4>};                             \
      case 5: return {k_tc_corr<QV, 5>, k_tc_accum<QV, 5>};                             \
      case 6: return {k_tc_corr<QV, 6>, k_tc_accum<QV, 6>};                             \
      default: return {nullptr, nullptr};                                               \
    }                                                                                   \
  }                                                                                     \
  }
