// CTA-cooperative EM sweep over batches of BI images (rows of Q = 2 QH coefficients).
//
// A persistent CTA (one per SM) streams batches of BI consecutive images through an
// NS-stage shared-memory ring (one bulk copy per image, slots padded to an odd number
// of 16-byte words) and works on a batch in barrier-separated phases whose work items
// put the image on the fastest-varying thread index, so that x and twiddle loads are
// broadcasts and each image's values sit in distinct banks.
//
// Log-weights are formed relative to a reference rotation p of each image, as
// differences over distance units {p + d, p - d} of the window:
//     S(p +- d) - S(p) = Re sum_k c'_k (e^{-+ i k 2 pi d / L} - 1),  c'_k = c_k e^{-i k theta_p},
// with a table of (cos - 1, -sin) computed in FP64 (cos - 1 = -2 sin^2), so the FP32
// values near the reference carry no rounding of the large common part 2 beta S(p).
//
//   correlation  item (k, i):  c_ik = sum_q conj(y_ikq) x_kq, rotated to the first reference
//                               (the window index of rotation 0, theta_hat_i folded in)
//   pass 1       item (d, i):  log-weights relative to the first reference
//   peak         warp i:       p_i = argmax; the distance D_i holding every log-weight above
//                               max - 40; c rotated to p_i; far log-weights re-referenced
//   pass 2       item (d, i):  log-weights within D_i recomputed relative to p_i
//   normalise    warp i:       w_il = exp(s_il - s_ip) / Z; per unit (w_+ + w_-, w_- - w_+)
//   back         item (k, i):  W_ik = e^{+i k theta_p} (1 + sum_{d <= D_i} (w_+ + w_-)(cos - 1)
//                                                         + i (w_- - w_+)(-sin))
//                               (the weights sum to 1; those beyond D_i are below e^-40 of the peak)
//   accumulate   thread (k, p): num_kq += sum_i W_ik y_ikq for two float4 columns of row k
//
// The distance-unit table sits in shared memory, or (TDG, for windows whose table does not fit
// next to the ring) stays in global memory, read through the read-only path: the (unit, image)
// items put the images on the fastest thread index, so a warp's table loads cover a few units and
// serve all of its images.
//
// Packed FP32 FMAs (f32x2) carry (re, im) pairs.  Per-thread FP32 column sums are folded
// into FP64 every 32 batches; the CTA writes FP64 partials [column][CTA] at the end, in the
// same layout as the other sweeps.
#pragma once
#include "common.cuh"

namespace mra {


// window indices of distance unit d around the reference p (-1 where absent)
__device__ __forceinline__ int2 unit_pair(int p, int d, int Lw, int L, bool wrap) {
  if (wrap) {
    int a = p + d;
    if (a >= L) a -= L;
    int b = p - d;
    if (b < 0) b += L;
    return make_int2(a, (d == 0 || 2 * d == L) ? -1 : b);
  }
  return make_int2(p + d < Lw ? p + d : -1, (d > 0 && p - d >= 0) ? p - d : -1);
}

template <int QH, int BI, int YF, bool TDG = false>
__global__ void __launch_bounds__(kV3Threads, 1) k_sweep_v3(const SweepV3Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = kV3Threads;
  constexpr int NW = NT / 32;
  constexpr int PH = QH / 2;      // float4 column pairs per row
  constexpr int ISTEP = NT / BI;  // item stride of the (row or unit, image) phases
  static_assert(QH % 2 == 0, "rows are handled as pairs of float4 columns");
  if (a.ctrl->done) return;
  const bool want_ysq = (a.ctrl->iter == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Kp1 = a.Kp1, L = a.L, Lw = a.Lw, M = a.M, NS = a.ns;
  const int cp = a.cp, sp = a.sp, dp = a.dp;
  const int r0 = a.r0, D1 = a.d1;
  const bool wrap = a.wrap != 0;
  const size_t slot = a.slot_bytes;

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);                      // [NS]
  unsigned char* ring = smem + a.off_ring;                                // [NS][BI][slot]
  const float4* xs4 = reinterpret_cast<const float4*>(smem + a.off_x);   // [M/2]  (x.re, x.im) pairs
  const float4* xr4 = reinterpret_cast<const float4*>(smem + a.off_xr);  // [M/2]  (x.im, -x.re) pairs
  const float2* td = TDG ? a.td : reinterpret_cast<const float2*>(smem + a.off_td);  // [Kp1][tdp]
  const int tdp = TDG ? a.nd : dp;
  auto tld = [&](const float2* t, int i) {
    if constexpr (TDG) return __ldg(t + i);
    else return t[i];
  };
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);  // [L]
  const float* lrs = reinterpret_cast<const float*>(smem + a.off_lr);    // [Lw]
  float2* cbuf = reinterpret_cast<float2*>(smem + a.off_c);              // [BI][cp]: c, later W
  float* sbuf = reinterpret_cast<float*>(smem + a.off_s);                // [BI][sp]: s, later w
  float2* w2 = reinterpret_cast<float2*>(smem + a.off_w2);               // [BI][dp]
  int4* info = reinterpret_cast<int4*>(smem + a.off_info);               // [BI] (phase, p, D, pass 2 bound)
  float* wlw = reinterpret_cast<float*>(smem + a.off_wl);                // [NW][sp]

  // ---- shared tables
  {
    float4* xw = reinterpret_cast<float4*>(smem + a.off_x);
    float4* xrw = reinterpret_cast<float4*>(smem + a.off_xr);
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
    for (int i = tid; i < M / 2; i += NT) {
      const float4 v = xg[i];
      xw[i] = v;
      xrw[i] = make_float4(v.y, -v.x, v.w, -v.z);
    }
    if constexpr (!TDG) {
      float2* tw = reinterpret_cast<float2*>(smem + a.off_td);
      for (int idx = tid; idx < Kp1 * dp; idx += NT) {
        const int k = idx / dp, d = idx - k * dp;
        tw[idx] = d < a.nd ? a.td[k * a.nd + d] : make_float2(0.f, 0.f);
      }
    }
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    float* lrw = reinterpret_cast<float*>(smem + a.off_lr);
    for (int i = tid; i < Lw; i += NT) lrw[i] = a.logrho32[i];
    for (int i = tid; i < NW * sp; i += NT) wlw[i] = 0.f;
    if (tid < NS) mbar_init(&bar[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();

  const int G = gridDim.x;
  const int nbatch = (a.N + BI - 1) / BI;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  auto issue = [&](int b, int st) {  // thread 0 only
    const int i0 = b * BI;
    const int nv = min(BI, a.N - i0);
    mbar_arrive_expect_tx(&bar[st], (uint32_t)nv * img_bytes);
    unsigned char* dst = ring + (size_t)st * BI * slot;
    for (int i = 0; i < nv; ++i) bulk_g2s(dst + (size_t)i * slot, a.y + (size_t)(i0 + i) * M, img_bytes, &bar[st]);
  };
  if (tid == 0)
    for (int j = 0; j < NS; ++j)
      if ((int)blockIdx.x + j * G < nbatch) issue(blockIdx.x + j * G, j);

  // accumulator thread (k, p) owns float4 columns k QH + p and k QH + p + PH of row k;
  // P = sum Re(W) y and R = sum Im(W) y give num = (P.re - R.im, P.im + R.re)
  const bool acc_on = tid < Kp1 * PH;
  const int ak = acc_on ? tid / PH : 0;
  const int af0 = ak * QH + (tid - ak * PH);
  float2 P[4], R[4];  // (P0.xy, P0.zw, P1.xy, P1.zw) and likewise for R
#pragma unroll
  for (int t = 0; t < 4; ++t) P[t] = R[t] = make_float2(0.f, 0.f);
  double acc64[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc64[t] = 0.0;
  auto fold = [&]() {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      acc64[2 * t] += (double)P[t].x - (double)R[t].y;
      acc64[2 * t + 1] += (double)P[t].y + (double)R[t].x;
      P[t] = R[t] = make_float2(0.f, 0.f);
    }
  };
  double ll_acc = 0.0, ysq_acc = 0.0;
  const float two_beta = a.two_beta;
  const int ii = tid % BI;  // image of this thread's (row, image) items
  const int it0 = tid / BI;
  const bool item_on = tid < ISTEP * BI;
  // forward items (unit, image): fsplit = 2 puts two adjacent threads on one item (even / odd rows)
  const int fsh = a.fsplit - 1;
  const int fit = tid >> fsh, fsub = tid & fsh;
  const int fstep = (NT >> fsh) / BI;
  const bool f_on = fit < fstep * BI;
  const int fii = fit % BI, fd0 = fit / BI;
  const unsigned fmask = fsh ? (3u << (lane & ~1)) : (1u << lane);

  // log-weights of the distance units d = fd0, fd0 + fstep, ... <= dmax around p (items (d, i))
  auto forward = [&](const float2* cr, float* srow, int p, int dmax) {
    for (int d = fd0; d <= dmax; d += fstep) {
      float2 ab0 = make_float2(0.f, 0.f), ab1 = ab0;  // (A', B) over two interleaved row sets
      const float2* tcol = td + d;
      const int kst = 2 << fsh;
      int k = fsub;
      for (; k + (kst >> 1) < Kp1; k += kst) {
        ab0 = __ffma2_rn(cr[k], tld(tcol, k * tdp), ab0);
        ab1 = __ffma2_rn(cr[k + (kst >> 1)], tld(tcol, (k + (kst >> 1)) * tdp), ab1);
      }
      if (k < Kp1) ab0 = __ffma2_rn(cr[k], tld(tcol, k * tdp), ab0);
      float A = ab0.x + ab1.x, B = ab0.y + ab1.y;
      if (fsh) {
        A += __shfl_xor_sync(fmask, A, 1);
        B += __shfl_xor_sync(fmask, B, 1);
      }
      if (fsub == 0) {
        const int2 ab = unit_pair(p, d, Lw, L, wrap);
        if (ab.x >= 0) srow[ab.x] = fmaf(two_beta, A - B, lrs[ab.x]);
        if (ab.y >= 0) srow[ab.y] = fmaf(two_beta, A + B, lrs[ab.y]);
      }
    }
  };

  // shift of image tid of the next batch, loaded one batch ahead
  auto load_shift = [&](int b) {
    const int i = b * BI + tid;
    return (a.shift && tid < BI && b < nbatch && i < a.N) ? a.shift[i] : 0;
  };
  int shift_next = load_shift(blockIdx.x);
  int n = 0;
  for (int b = blockIdx.x; b < nbatch; b += G, ++n) {
    const int st = n % NS;
    const uint32_t parity = (uint32_t)((n / NS) & 1);
    const bool ok = mbar_wait_bounded(&bar[st], parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        // let the copies still in flight land before the CTA exits: batches n .. n + NS - 2
        // (n + NS - 1 at the first batch, whose stages the prologue filled)
        const int last = n == 0 ? NS - 1 : n + NS - 2;
        for (int j = n; j <= last && b + (j - n) * G < nbatch; ++j)
          mbar_wait_bounded(&bar[j % NS], (uint32_t)((j / NS) & 1));
      }
      break;
    }
    const int i0 = b * BI;
    const int nv = min(BI, a.N - i0);
    const unsigned char* stage = ring + (size_t)st * BI * slot;
    if (tid < BI) {
      int ph = (shift_next % L + a.phase0) % L;
      if (ph < 0) ph += L;
      info[tid] = make_int4(ph, r0, D1, D1);
      shift_next = load_shift(b + G);
    }
    __syncthreads();
    // every thread finished batch n - 1 before the first barrier above, so its stage can
    // take batch n + NS - 1: lanes of the last warp issue one copy each
    if (warp == NW - 1 && n > 0 && b + (NS - 1) * G < nbatch) {
      const int bn = b + (NS - 1) * G, stn = (n - 1) % NS;
      const int nvn = min(BI, a.N - bn * BI);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) mbar_arrive_expect_tx(&bar[stn], (uint32_t)nvn * img_bytes);
      __syncwarp();
      for (int i = lane; i < nvn; i += 32)
        bulk_g2s(ring + ((size_t)stn * BI + i) * slot, a.y + (size_t)(bn * BI + i) * M, img_bytes, &bar[stn]);
    }

    // ---- correlation, items (k, i)
    if (item_on && ii < nv) {
      const float4* yimg = reinterpret_cast<const float4*>(stage + (size_t)ii * slot);
      const int ph = info[ii].x;
      for (int k = it0; k < Kp1; k += ISTEP) {
        // Re c = sum (y.re x.re + y.im x.im), Im c = sum (y.re x.im - y.im x.re)
        float2 p0 = make_float2(0.f, 0.f), p1 = p0, q0 = p0, q1 = p0;
        float sq0 = 0.f, sq1 = 0.f;
        const float4* yr = yimg + k * QH;
        const float4* xr = xs4 + k * QH;
        const float4* xq = xr4 + k * QH;
#pragma unroll
        for (int p = 0; p < QH; ++p) {
          const float4 yv = load_y4<YF>(yr, p), xv = xr[p], xw = xq[p];
          const float2 ya = make_float2(yv.x, yv.y), yb = make_float2(yv.z, yv.w);
          p0 = __ffma2_rn(ya, make_float2(xv.x, xv.y), p0);
          p1 = __ffma2_rn(yb, make_float2(xv.z, xv.w), p1);
          q0 = __ffma2_rn(ya, make_float2(xw.x, xw.y), q0);
          q1 = __ffma2_rn(yb, make_float2(xw.z, xw.w), q1);
          if (want_ysq) {
            sq0 = fmaf(yv.x, yv.x, sq0); sq1 = fmaf(yv.y, yv.y, sq1);
            sq0 = fmaf(yv.z, yv.z, sq0); sq1 = fmaf(yv.w, yv.w, sq1);
          }
        }
        float2 c = make_float2((p0.x + p0.y) + (p1.x + p1.y), (q0.x + q0.y) + (q1.x + q1.y));
        if (ph != 0) c = cmul(c, tfs[(k * ph) % L]);
        if (a.tw) c = cmul(c, a.tw[k * a.twp + r0]);  // dense window: the first reference's angle
        cbuf[ii * cp + k] = c;
        if (want_ysq) ysq_acc += (double)(sq0 + sq1);
      }
    }
    __syncthreads();

    // ---- pass 1 relative to the first reference r0
    if (f_on && fii < nv) forward(cbuf + fii * cp, sbuf + fii * sp, r0, D1);
    __syncthreads();

    // ---- peak, significant distance, rotation to the peak; warp per image
    for (int i = warp; i < nv; i += NW) {
      float* srow = sbuf + i * sp;
      float bv = -INFINITY;
      int bl = 0x7fffffff;
      for (int l = lane; l < Lw; l += 32) {
        const float v = srow[l];
        if (v > bv) bv = v, bl = l;
      }
      // argmax with the smallest index among ties: order-preserving integer keys of the values
      const uint32_t u = __float_as_uint(bv);
      const uint32_t key = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
      const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
      int p = (int)__reduce_min_sync(0xffffffffu, key == kmax ? (uint32_t)bl : 0xffffffffu);
      if (p >= Lw) p = r0;  // every log-weight is -inf
      const float thr = srow[p] - 40.f;
      uint32_t dist = 0;
      for (int l = lane; l < Lw; l += 32) {
        if (srow[l] >= thr) {
          int dd = l > p ? l - p : p - l;
          if (wrap && 2 * dd > L) dd = L - dd;
          dist = max(dist, (uint32_t)dd);
        }
      }
      dist = __reduce_max_sync(0xffffffffu, dist);
      const int ph1 = info[i].x;
      if (p != r0) {
        // values beyond the pass 2 range: shift pass 1 to the new reference
        const float shiftv = srow[p] - lrs[p];
        __syncwarp();
        for (int l = lane; l < Lw; l += 32) srow[l] -= shiftv;
        if (a.tw) {  // dense window: p - r0 window steps, from the distance-unit table
          const int dr = p - r0, ad = dr < 0 ? -dr : dr;
          for (int k = lane; k < Kp1; k += 32)
            cbuf[i * cp + k] = cmul(cbuf[i * cp + k], td_rot(tld(td, k * tdp + ad), dr));
          if (lane == 0) info[i] = make_int4(ph1, p, (int)dist, (int)dist);
        } else {
          int dr = (p - r0) % L;
          if (dr < 0) dr += L;
          for (int k = lane; k < Kp1; k += 32) cbuf[i * cp + k] = cmul(cbuf[i * cp + k], tfs[(k * dr) % L]);
          if (lane == 0) info[i] = make_int4((ph1 + dr) % L, p, (int)dist, (int)dist);
        }
      } else if (lane == 0) {
        info[i] = make_int4(ph1, p, (int)dist, -1);
      }
    }
    __syncthreads();

    // ---- pass 2 relative to the peak, only where it moved
    if (f_on && fii < nv) {
      const int4 f = info[fii];
      forward(cbuf + fii * cp, sbuf + fii * sp, f.y, f.w);
    }
    __syncthreads();

    // ---- normalisation, one warp per image
    for (int i = warp; i < nv; i += NW) {
      float* srow = sbuf + i * sp;
      const int4 f = info[i];
      const int p = f.y;
      const float m = srow[p];
      float z = 0.f, s0 = 0.f;
      for (int l = lane; l < Lw; l += 32) {
        const float e = __expf(srow[l] - m);
        srow[l] = e;
        z += e;
      }
      for (int k = lane; k < Kp1; k += 32) s0 += cbuf[i * cp + k].x;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        z += __shfl_xor_sync(0xffffffffu, z, o);
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      }
      const float inv = __frcp_rn(z);
      float* wl = wlw + warp * sp;
      float* wo = a.w_out ? a.w_out + (size_t)(i0 + i) * Lw : nullptr;
      for (int l = lane; l < Lw; l += 32) {
        const float w = srow[l] * inv;
        srow[l] = w;
        wl[l] += w;
        if (wo) wo[l] = w;
      }
      __syncwarp();
      for (int d = lane; d <= f.z; d += 32) {
        const int2 ab = unit_pair(p, d, Lw, L, wrap);
        const float wa = ab.x >= 0 ? srow[ab.x] : 0.f, wb = ab.y >= 0 ? srow[ab.y] : 0.f;
        w2[i * dp + d] = make_float2(wa + wb, wb - wa);
      }
      if (lane == 0) ll_acc += (double)fmaf(two_beta, s0, m + __logf(z));
    }
    __syncthreads();

    // ---- back transform, items (k, i); W replaces c
    if (item_on && ii < nv) {
      const float2* wr = w2 + ii * dp;
      const int4 f = info[ii];
      for (int k = it0; k < Kp1; k += ISTEP) {
        float2 v0 = make_float2(0.f, 0.f), v1 = v0;
        const float2* trow = td + k * tdp;
        int d = 0;
        for (; d + 1 <= f.z; d += 2) {
          v0 = __ffma2_rn(wr[d], tld(trow, d), v0);
          v1 = __ffma2_rn(wr[d + 1], tld(trow, d + 1), v1);
        }
        if (d <= f.z) v0 = __ffma2_rn(wr[d], tld(trow, d), v0);
        float2 W = make_float2(1.f + (v0.x + v1.x), v0.y + v1.y);
        if (f.x != 0) W = cmul_conj_b(W, tfs[(k * f.x) % L]);
        if (a.tw) W = cmul_conj_b(W, a.tw[k * a.twp + f.y]);  // dense window: the reference's angle
        cbuf[ii * cp + k] = W;
      }
    }
    __syncthreads();

    // ---- accumulate W_ik y_ikq
    if (acc_on) {
#pragma unroll 4
      for (int i = 0; i < nv; ++i) {
        const float4* y4 = reinterpret_cast<const float4*>(stage + (size_t)i * slot);
        const float4 ya = load_y4<YF>(y4, af0), yb = load_y4<YF>(y4, af0 + PH);
        const float2 w = cbuf[i * cp + ak];
        const float2 wre = make_float2(w.x, w.x), wim = make_float2(w.y, w.y);
        const float2 yv[4] = {make_float2(ya.x, ya.y), make_float2(ya.z, ya.w), make_float2(yb.x, yb.y),
                              make_float2(yb.z, yb.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          P[t] = __ffma2_rn(wre, yv[t], P[t]);
          R[t] = __ffma2_rn(wim, yv[t], R[t]);
        }
      }
      if ((n & 31) == 31) fold();
    }
    // the next batch's first barrier orders these reads before the stage is refilled
  }
  if (acc_on) fold();

  // ---- FP64 partials, column-major [col][G] with col = 4 (float4 column) + component
  const int cta = blockIdx.x;
  if (acc_on) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      a.part[(size_t)(4 * af0 + t) * G + cta] = acc64[t];
      a.part[(size_t)(4 * (af0 + PH) + t) * G + cta] = acc64[4 + t];
    }
  }
  __syncthreads();
  for (int l = tid; l < Lw; l += NT) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += (double)wlw[w * sp + l];
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

// Instantiation table for one row width QH (float4 per row): batches of 16, 12, 8 or 4
// images, y in FP32 (yf = 0) or as the BF16 hi/lo split (yf = 1); sweep_v3g_qh* holds the
// instances that read the distance-unit table from global memory (batches of 8 or 4).
#define MRA_SWEEP_V3_TABLE(QH)                                     \
  namespace mra {                                                  \
  SweepV3Fn sweep_v3_qh##QH(int bi, int yf) {                      \
    switch (bi * 2 + (yf ? 1 : 0)) {                               \
      case 32: return k_sweep_v3<QH, 16, 0>;                       \
      case 33: return k_sweep_v3<QH, 16, 1>;                       \
      case 24: return k_sweep_v3<QH, 12, 0>;                       \
      case 25: return k_sweep_v3<QH, 12, 1>;                       \
      case 16: return k_sweep_v3<QH, 8, 0>;                        \
      case 17: return k_sweep_v3<QH, 8, 1>;                        \
      case 8: return k_sweep_v3<QH, 4, 0>;                         \
      case 9: return k_sweep_v3<QH, 4, 1>;                         \
      default: return nullptr;                                     \
    }                                                              \
  }                                                                \
  SweepV3Fn sweep_v3g_qh##QH(int bi, int yf) {                     \
    switch (bi * 2 + (yf ? 1 : 0)) {                               \
      case 16: return k_sweep_v3<QH, 8, 0, true>;                  \
      case 17: return k_sweep_v3<QH, 8, 1, true>;                  \
      case 8: return k_sweep_v3<QH, 4, 0, true>;                   \
      case 9: return k_sweep_v3<QH, 4, 1, true>;                   \
      default: return nullptr;                                     \
    }                                                              \
  }                                                                \
  }
