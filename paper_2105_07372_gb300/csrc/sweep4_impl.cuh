// Chunked two-read EM sweep (rows of Q a multiple of 8).
//
// A persistent CTA takes chunks of C consecutive images.  For each chunk:
//
//   read 1 (warp per image)   every warp streams its images of the chunk through a one-slot
//                             shared-memory ring (bulk copy, mbarrier completion, L2 evict_last
//                             hint) and forms c_ik = sum_q conj(y_ikq) x_kq with the quad layout
//                             of the warp sweep (quad r owns rows k = r (mod 8), lane j float4
//                             columns j, j+4, ...), rotated to the first reference of the window;
//                             c goes to a per-chunk buffer, y is not kept
//   transforms (CTA)          on the whole chunk at once, images on the fastest thread index:
//                             pass 1 relative to the first reference, peak and significant
//                             distance (warp per image), pass 2 relative to the peak,
//                             normalisation (warp per image), back transform -> W_ik
//   read 2 (warp per image)   the same images again (now from L2, evict_first hint):
//                             num_kq += W_ik y_ikq into per-lane FP32 registers
//
// Reading y twice keeps it out of shared memory during the transforms, so a chunk of
// 32..128 images gives the transform phases enough parallel work, while only one image
// per warp occupies the ring.  The log-weight arithmetic is the batch sweep's
// (sweep3_impl.cuh): differences over distance units around a reference rotation with
// an FP64-built (cos - 1, -sin) table.
#pragma once
#include "common.cuh"
#include "sweep3_impl.cuh"

namespace mra {

// Per-lane accumulators above 64 floats need more than 128 registers: 256 threads, one CTA per SM.
template <int QV, int MR>
struct SweepV4Shape {
  static constexpr bool kBig = MR * QV * 4 > 64;
};

__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// bulk copy global -> shared with an L2 cache policy (addresses and size multiples of 16)
__device__ __forceinline__ void bulk_g2s_hint(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

template <int QV, int MR, int NTH, int MINB, int YF>
__global__ void __launch_bounds__(NTH, MINB) k_sweep_v4(const SweepV4Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = NTH;
  constexpr int NW = NT / 32;
  constexpr int row4 = QV * 4;  // float4 per row
  if (a.ctrl->done) return;
  const bool want_ysq = (a.ctrl->iter == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = lane >> 2, j = lane & 3;
  const int Kp1 = a.Kp1, L = a.L, Lw = a.Lw, M = a.M;
  const int cp = a.cp, sp = a.sp, dp = a.dp;
  const int r0 = a.r0, D1 = a.d1;
  const bool wrap = a.wrap != 0;
  const int C = 1 << a.lc;  // images per chunk

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);                    // [NW]
  unsigned char* slot = smem + a.off_ring + (size_t)warp * a.slot_bytes;  // this warp's slot
  const float4* xs4 = reinterpret_cast<const float4*>(smem + a.off_x);  // [M/2]
  const float2* td = reinterpret_cast<const float2*>(smem + a.off_td);  // [Kp1][dp]
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);  // [L]
  const float* lrs = reinterpret_cast<const float*>(smem + a.off_lr);   // [Lw]
  float2* cbuf = reinterpret_cast<float2*>(smem + a.off_c);             // [C][cp]: c, later W
  float* sbuf = reinterpret_cast<float*>(smem + a.off_s);               // [C][sp]
  float2* w2 = reinterpret_cast<float2*>(smem + a.off_w2);              // [C][dp]
  int4* info = reinterpret_cast<int4*>(smem + a.off_info);              // [C] (phase, p, D, pass 2 bound)
  float* wlw = reinterpret_cast<float*>(smem + a.off_wl);               // [4 NW][sp]: W[l] per 8-lane group

  {
    float4* xw = reinterpret_cast<float4*>(smem + a.off_x);
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
    for (int i = tid; i < M / 2; i += NT) xw[i] = xg[i];
    float2* tw = reinterpret_cast<float2*>(smem + a.off_td);
    for (int idx = tid; idx < Kp1 * dp; idx += NT) {
      const int k = idx / dp, d = idx - k * dp;
      tw[idx] = d < a.nd ? a.td[k * a.nd + d] : make_float2(0.f, 0.f);
    }
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    float* lrw = reinterpret_cast<float*>(smem + a.off_lr);
    for (int i = tid; i < Lw; i += NT) lrw[i] = a.logrho32[i];
    for (int i = tid; i < 4 * NW * sp; i += NT) wlw[i] = 0.f;
    if (tid < NW) mbar_init(&bar[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();

  const int G = gridDim.x;
  const int nchunk = (a.N + C - 1) / C;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  const uint64_t pol_keep = l2_policy_evict_last(), pol_drop = l2_policy_evict_first();
  uint64_t* mybar = &bar[warp];
  // this warp's images of chunk ch: local indices warp, warp + NW, ... below nv
  auto count = [&](int ch) {
    const int nv = min(C, a.N - ch * C);
    return warp < nv ? (nv - warp + NW - 1) / NW : 0;
  };
  auto issue = [&](int ch, int t, bool second) {  // lane 0
    const int img = ch * C + warp + t * NW;
    mbar_arrive_expect_tx(mybar, img_bytes);
    bulk_g2s_hint(slot, a.y + (size_t)img * M, img_bytes, mybar, second ? pol_drop : pol_keep);
  };
  // the next load after (chunk n, item t of read `second`): returns false when there is none
  auto issue_next = [&](int n, int t, bool second) {
    const int ch = blockIdx.x + n * G;
    const int cnt = count(ch);
    if (t + 1 < cnt) {
      issue(ch, t + 1, second);
      return true;
    }
    if (!second) {
      issue(ch, 0, true);
      return true;
    }
    for (int m = n + 1; blockIdx.x + m * G < nchunk; ++m)
      if (count(blockIdx.x + m * G) > 0) {
        issue(blockIdx.x + m * G, 0, false);
        return true;
      }
    return false;
  };

  float4 acc[MR][QV];
#pragma unroll
  for (int m = 0; m < MR; ++m)
#pragma unroll
    for (int u = 0; u < QV; ++u) acc[m][u] = make_float4(0.f, 0.f, 0.f, 0.f);
  double ll_acc = 0.0, ysq_acc = 0.0;
  const float two_beta = a.two_beta;
  uint32_t uses = 0;     // completed phases of this warp's mbarrier
  bool pending = false;  // a load of this warp is in flight
  bool failed = false;

  {
    int first = -1;
    for (int m = 0; (int)blockIdx.x + m * G < nchunk; ++m)
      if (count(blockIdx.x + m * G) > 0) {
        first = m;
        break;
      }
    pending = first >= 0;
    if (pending && lane == 0) issue(blockIdx.x + first * G, 0, false);
  }

  // wait for this warp's slot; on expiry record the status and stop streaming
  auto wait_slot = [&]() {
    const bool ok = mbar_wait_bounded(mybar, uses & 1u);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
      failed = true;
      return false;
    }
    ++uses;
    pending = false;
    return true;
  };

  int n = 0;
  for (int ch = blockIdx.x; ch < nchunk; ch += G, ++n) {
    const int nv = min(C, a.N - ch * C);
    const int cnt = count(ch);
    // ---- read 1: correlation, warp per image
    for (int t = 0; t < cnt && !failed; ++t) {
      if (!wait_slot()) break;
      const int li = warp + t * NW;
      const int img = ch * C + li;
      const float4* y4 = reinterpret_cast<const float4*>(slot);
      int sj = 0;
      if (a.shift) {
        sj = a.shift[img] % L;
        if (sj < 0) sj += L;
      }
      const int ph = (sj + a.phase0) % L;  // rotation to the first reference
      float sq = 0.f;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const int k = r + 8 * m;
        float cr = 0.f, ci = 0.f;
        if (k < Kp1) {
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const int pidx = k * row4 + j + 4 * u;
            const float4 xv = xs4[pidx];
            const float4 yv = load_y4<YF>(y4, pidx);
            cr = fmaf(yv.x, xv.x, cr); cr = fmaf(yv.y, xv.y, cr);
            ci = fmaf(yv.x, xv.y, ci); ci = fmaf(-yv.y, xv.x, ci);
            cr = fmaf(yv.z, xv.z, cr); cr = fmaf(yv.w, xv.w, cr);
            ci = fmaf(yv.z, xv.w, ci); ci = fmaf(-yv.w, xv.z, ci);
            if (want_ysq) {
              sq = fmaf(yv.x, yv.x, sq); sq = fmaf(yv.y, yv.y, sq);
              sq = fmaf(yv.z, yv.z, sq); sq = fmaf(yv.w, yv.w, sq);
            }
          }
        }
        cr += __shfl_xor_sync(0xffffffffu, cr, 1);
        ci += __shfl_xor_sync(0xffffffffu, ci, 1);
        cr += __shfl_xor_sync(0xffffffffu, cr, 2);
        ci += __shfl_xor_sync(0xffffffffu, ci, 2);
        if (j == 0 && k < Kp1) {
          float2 c = make_float2(cr, ci);
          if (ph != 0) c = cmul(c, tfs[(k * ph) % L]);
          if (a.tw) c = cmul(c, a.tw[k * a.twp + r0]);  // dense window: the first reference's angle
          cbuf[li * cp + k] = c;
        }
      }
      if (want_ysq) {
        sq = warp_sum(sq);
        if (lane == 0) ysq_acc += (double)sq;
      }
      if (lane == 0) info[li] = make_int4(ph, r0, D1, D1);
      // the slot is free once every lane has read it
      __syncwarp();
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        pending = issue_next(n, t, false);
      }
      pending = __shfl_sync(0xffffffffu, (int)pending, 0);
    }
    if (__syncthreads_or(failed)) break;

    // ---- transforms on the chunk (images on the fastest thread index)
    {
      // pass 1: items (d, i)
      const int step = NT / C;  // C divides NT
      const int ii = tid & (C - 1), d0 = tid >> a.lc;
      // this thread's units d = d0 + step u (u < kU) of image i: each c_k load serves all of them
      constexpr int kU = 4;
      auto forward = [&](int i, int p, int dmax) {
        const float2* cr = cbuf + i * cp;
        float* srow = sbuf + i * sp;
        for (int db = d0; db <= dmax; db += kU * step) {
          float2 ab[kU][2];
#pragma unroll
          for (int u = 0; u < kU; ++u) ab[u][0] = ab[u][1] = make_float2(0.f, 0.f);
          int k = 0;
          for (; k + 1 < Kp1; k += 2) {
            const float2 c0 = cr[k], c1 = cr[k + 1];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              const int d = min(db + u * step, dmax);  // past dmax: a repeat, not stored
              ab[u][0] = __ffma2_rn(c0, td[k * dp + d], ab[u][0]);
              ab[u][1] = __ffma2_rn(c1, td[(k + 1) * dp + d], ab[u][1]);
            }
          }
          if (k < Kp1) {
            const float2 c0 = cr[k];
#pragma unroll
            for (int u = 0; u < kU; ++u) ab[u][0] = __ffma2_rn(c0, td[k * dp + min(db + u * step, dmax)], ab[u][0]);
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int d = db + u * step;
            if (d <= dmax) {
              const float A = ab[u][0].x + ab[u][1].x, B = ab[u][0].y + ab[u][1].y;
              const int2 pr = unit_pair(p, d, Lw, L, wrap);
              if (pr.x >= 0) srow[pr.x] = fmaf(two_beta, A - B, lrs[pr.x]);
              if (pr.y >= 0) srow[pr.y] = fmaf(two_beta, A + B, lrs[pr.y]);
            }
          }
        }
      };
      if (ii < nv) forward(ii, r0, D1);
      __syncthreads();
      // peak, significant distance, rotation of c to the peak: 8 lanes per image, four
      // images per warp at a time (xor shuffles below 8 stay inside a group)
      const int grp = lane >> 3, sub = lane & 7;
      for (int i0 = warp * 4; i0 < nv; i0 += 4 * NW) {
        const int i = min(i0 + grp, nv - 1);  // groups past the end repeat the last image, without writes
        const bool own = i0 + grp < nv;
        float* srow = sbuf + i * sp;
        float bv = -INFINITY;
        int bl = 0x7fffffff;
        for (int l = sub; l < Lw; l += 8) {
          const float v = srow[l];
          if (v > bv) bv = v, bl = l;
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
          if (ov > bv || (ov == bv && ol < bl)) bv = ov, bl = ol;
        }
        const int p = bl < Lw ? bl : r0;  // every log-weight -inf: keep the first reference
        const float thr = srow[p] - 40.f;
        int dist = 0;
        for (int l = sub; l < Lw; l += 8) {
          if (srow[l] >= thr) {
            int dd = l > p ? l - p : p - l;
            if (wrap && 2 * dd > L) dd = L - dd;
            dist = max(dist, dd);
          }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) dist = max(dist, __shfl_xor_sync(0xffffffffu, dist, o));
        const int ph1 = info[i].x;
        const float shiftv = srow[p] - lrs[p];
        __syncwarp();
        if (own) {
          if (p != r0) {
            for (int l = sub; l < Lw; l += 8) srow[l] -= shiftv;
            if (a.tw) {  // dense window: p - r0 window steps, from the distance-unit table
              const int dr = p - r0, ad = dr < 0 ? -dr : dr;
              for (int k = sub; k < Kp1; k += 8) cbuf[i * cp + k] = cmul(cbuf[i * cp + k], td_rot(td[k * dp + ad], dr));
              if (sub == 0) info[i] = make_int4(ph1, p, dist, dist);
            } else {
              int dr = (p - r0) % L;
              if (dr < 0) dr += L;
              for (int k = sub; k < Kp1; k += 8) cbuf[i * cp + k] = cmul(cbuf[i * cp + k], tfs[(k * dr) % L]);
              if (sub == 0) info[i] = make_int4((ph1 + dr) % L, p, dist, dist);
            }
          } else if (sub == 0) {
            info[i] = make_int4(ph1, p, dist, -1);
          }
        }
        __syncwarp();
      }
      __syncthreads();
      if (ii < nv) {
        const int4 f = info[ii];
        forward(ii, f.y, f.w);
      }
      __syncthreads();
      // normalisation: 8 lanes per image, four images per warp at a time
      for (int i0 = warp * 4; i0 < nv; i0 += 4 * NW) {
        const int i = min(i0 + grp, nv - 1);
        const bool own = i0 + grp < nv;
        float* srow = sbuf + i * sp;
        const int4 f = info[i];
        const int p = f.y;
        const float mref = srow[p];
        float z = 0.f, s0 = 0.f;
        for (int l = sub; l < Lw; l += 8) z += __expf(srow[l] - mref);
        for (int k = sub; k < Kp1; k += 8) s0 += cbuf[i * cp + k].x;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          z += __shfl_xor_sync(0xffffffffu, z, o);
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        }
        const float inv = __frcp_rn(z);
        __syncwarp();
        if (own) {
          float* wo = a.w_out ? a.w_out + (size_t)(ch * C + i) * Lw : nullptr;
          float* wl = wlw + (warp * 4 + grp) * sp;  // this group's W[l] row
          for (int l = sub; l < Lw; l += 8) {
            const float w = __expf(srow[l] - mref) * inv;
            srow[l] = w;
            wl[l] += w;
            if (wo) wo[l] = w;
          }
        }
        __syncwarp();
        if (own) {
          for (int d = sub; d <= f.z; d += 8) {
            const int2 ab = unit_pair(p, d, Lw, L, wrap);
            const float wa = ab.x >= 0 ? srow[ab.x] : 0.f, wb = ab.y >= 0 ? srow[ab.y] : 0.f;
            w2[i * dp + d] = make_float2(wa + wb, wb - wa);
          }
          if (sub == 0) ll_acc += (double)fmaf(two_beta, s0, mref + __logf(z));
        }
      }
      __syncthreads();
      // back transform: items (k, i), rows k = d0 + step u of image i; each w2_d load serves all
      // of them; W replaces c
      if (ii < nv) {
        constexpr int kR = 6;
        const float2* wr = w2 + ii * dp;
        const int4 f = info[ii];
        for (int kb = d0; kb < Kp1; kb += kR * step) {
          float2 v[kR];
#pragma unroll
          for (int u = 0; u < kR; ++u) v[u] = make_float2(0.f, 0.f);
          for (int d = 0; d <= f.z; ++d) {
            const float2 wv = wr[d];
#pragma unroll
            for (int u = 0; u < kR; ++u) v[u] = __ffma2_rn(wv, td[min(kb + u * step, Kp1 - 1) * dp + d], v[u]);
          }
#pragma unroll
          for (int u = 0; u < kR; ++u) {
            const int k = kb + u * step;
            if (k < Kp1) {
              float2 W = make_float2(1.f + v[u].x, v[u].y);
              if (f.x != 0) W = cmul_conj_b(W, tfs[(k * f.x) % L]);
              if (a.tw) W = cmul_conj_b(W, a.tw[k * a.twp + f.y]);  // dense window: the reference's angle
              cbuf[ii * cp + k] = W;
            }
          }
        }
      }
      __syncthreads();
    }

    // ---- read 2: accumulation, warp per image (the same images, from L2)
    for (int t = 0; t < cnt && !failed; ++t) {
      if (!wait_slot()) break;
      const int li = warp + t * NW;
      const float4* y4 = reinterpret_cast<const float4*>(slot);
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const int k = r + 8 * m;
        if (k < Kp1) {
          const float2 w = cbuf[li * cp + k];
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const float4 yv = load_y4<YF>(y4, k * row4 + j + 4 * u);
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
        pending = issue_next(n, t, true);
      }
      pending = __shfl_sync(0xffffffffu, (int)pending, 0);
    }
  }
  // a load still in flight after a failure: let it land before the ring is reused
  if (pending && lane == 0) mbar_wait_bounded(mybar, uses & 1u);

  // ---- CTA combination: per-warp FP32 sums through the (now idle) ring, summed in FP64
  __syncthreads();
  float4* red4 = reinterpret_cast<float4*>(smem + a.off_ring + (size_t)warp * a.slot_bytes);  // [M/2]
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int k = r + 8 * m;
    if (k < Kp1) {
#pragma unroll
      for (int u = 0; u < QV; ++u) red4[k * row4 + j + 4 * u] = acc[m][u];
    }
  }
  __syncthreads();
  const int cta = blockIdx.x;
  for (int col = tid; col < 2 * M; col += NT) {
    double sum = 0.0;
    for (int w = 0; w < NW; ++w)
      sum += (double)reinterpret_cast<const float*>(smem + a.off_ring + (size_t)w * a.slot_bytes)[col];
    a.part[(size_t)col * G + cta] = sum;
  }
  for (int l = tid; l < Lw; l += NT) {
    double s = 0.0;
    for (int w = 0; w < 4 * NW; ++w) s += (double)wlw[w * sp + l];
    a.part[(size_t)(2 * M + l) * G + cta] = s;
  }
  __shared__ double red[2][NW];
  ll_acc = warp_sum_d(ll_acc);
  ysq_acc = warp_sum_d(ysq_acc);
  if (lane == 0) red[0][warp] = ll_acc, red[1][warp] = ysq_acc;
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < NW; ++w) t0 += red[0][w], t1 += red[1][w];
    a.part[(size_t)(2 * M + Lw) * G + cta] = t0;
    a.part[(size_t)(2 * M + Lw + 1) * G + cta] = t1;
  }
}

}  // namespace mra

// Instantiation table for one row width QV (float4 per lane per row) and y format YF: MR = 1..7
// rows per quad; one CTA of 512 threads or two of 256 per SM (256 threads and one CTA per SM for
// the largest per-lane accumulators).
#define MRA_SWEEP_V4_CASE(QV, MR, YF)                                                    \
  case MR:                                                                               \
    if (SweepV4Shape<QV, MR>::kBig)                                                      \
      return cpsm == 1 ? SweepV4Launch{k_sweep_v4<QV, MR, 256, 1, YF>, 256, 1}           \
                       : SweepV4Launch{nullptr, 0, 0};                                   \
    return cpsm == 1 ? SweepV4Launch{k_sweep_v4<QV, MR, 512, 1, YF>, 512, 1}             \
                     : SweepV4Launch{k_sweep_v4<QV, MR, 256, 2, YF>, 256, 2};
#define MRA_SWEEP_V4_TABLE(QV, YF)                           \
  namespace mra {                                            \
  SweepV4Launch sweep_v4_q##QV##_f##YF(int MR, int cpsm) {   \
    switch (MR) {                                            \
      MRA_SWEEP_V4_CASE(QV, 1, YF)                           \
      MRA_SWEEP_V4_CASE(QV, 2, YF)                           \
      MRA_SWEEP_V4_CASE(QV, 3, YF)                           \
      MRA_SWEEP_V4_CASE(QV, 4, YF)                           \
      MRA_SWEEP_V4_CASE(QV, 5, YF)                           \
      MRA_SWEEP_V4_CASE(QV, 6, YF)                           \
      MRA_SWEEP_V4_CASE(QV, 7, YF)                           \
      default: return {nullptr, 0, 0};                       \
    }                                                        \
  }                                                          \
  }
