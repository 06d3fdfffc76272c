// Lean warp-streaming EM sweep for grid windows of at most 32 mirror units (rows of Q a
// multiple of 8 coefficients), Eq. weights_2d_em and Eq. coefficients_update.
//
// The same work as the warp sweep (sweep_impl.cuh), arranged for fewer instructions per image:
//
//   correlation   quad layout as in the warp sweep (quad r owns rows k = r, r+8, ...; lane j of
//                 a quad owns the float4 columns j, j+4, ...), with packed FP32 FMAs: the two
//                 partial sums (y.re x.re, y.im x.im) and (y.re x.im, y.im x.re) of a complex
//                 pair accumulate in one f32x2 FMA each (the second against x with its parts
//                 swapped in registers; Im c is the difference of its two lanes)
//   pass 1        each lane owns one mirror unit {+o, -o} and sums over every row, reading c_k
//                 as a shared-memory broadcast; no cross-lane sums per unit.  The peak and the
//                 40-below cut come from two redux.sync each (floats mapped to ordered ints)
//   pass 2        as in the warp sweep: c rotated to the peak, the FP64-built (cos t - 1, -sin t)
//                 table, lane j of every quad taking the distance d = j (its table entries held
//                 in registers); the values are exact differences from the peak
//   sharp images  (every weight above e^-40 of the peak within 3 grid steps of it, the usual
//                 case) are normalised in registers and back-transformed over those distances
//                 in the "1 + sum" form; other images take the warp sweep's general path
//                 (a per-warp buffer over the window)
//   accumulate    num_kq += W_k y_kq into per-lane FP32 registers, combined per CTA in FP64
//
// Precision is that of the warp sweep: pass 1 only places the peak and the cut, pass 2 and the
// back transform work relative to the peak.
#pragma once
#include "common.cuh"

namespace mra {

template <int QV, int MR>
struct SweepV5Shape {
  static constexpr int kThreads = 512;
};
// Rows of the pass-1 tables in shared memory: K+1 padded to 8 MR with zero rows, so that the
// pass runs over a compile-time count without guards.

// Order-preserving maps between floats and ints (for redux.sync maxima of floats).
__device__ __forceinline__ int f2ord(float v) {
  const int i = __float_as_int(v);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__device__ __forceinline__ int mod_l(int a, int L, float invL) {
  int m = a - __float2int_rz((float)a * invL) * L;
  if (m < 0) m += L;
  if (m >= L) m -= L;
  return m;
}

// NUPC: the unit table's pitch (mirror units padded to 20 or 40), fixed at compile time.
// A device function of (arguments, CTA index, grid size), as the warp sweep: the batched persistent
// kernel runs it for one instance's CTA slot; k_sweep_v5 launches it directly.
template <int QV, int MR, int NUPC>
__device__ __forceinline__ void sweep_v5_body(const SweepV2Args& a, const int cta_, const int grid_) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = SweepV5Shape<QV, MR>::kThreads;
  constexpr int row4 = QV * 4;  // float4 per row
  constexpr unsigned FULL = 0xffffffffu;
  // the state (x, log rho, control words) may come from another CTA of a persistent launch: read
  // it through L2
  if (__ldcg(&a.ctrl->done)) return;
  const bool want_ysq = (__ldcg(&a.ctrl->iter) == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = a.nwarps;
  const int r = lane >> 2, j = lane & 3;
  const int Kp1 = a.Kp1, L = a.L, Lw = a.Lw, NU = a.NU, M = a.M;
  constexpr int NUP = NUPC, KR = 8 * MR;  // unit pitch, padded rows
  const float invL = 1.0f / (float)L;

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);  // [NT/32][2]
  unsigned char* ring = smem + a.off_ring;            // [nwarps][2][slot]
  const float4* xs4 = reinterpret_cast<const float4*>(smem + a.off_x);   // x
  const float2* tus = reinterpret_cast<const float2*>(smem + a.off_tu);  // [KR][NUP], rows >= K+1 zero
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);  // [L]
  const float* lrs = reinterpret_cast<const float*>(smem + a.off_lr);    // [Lw]
  const int2* uab = reinterpret_cast<const int2*>(smem + a.off_units);   // [NUP]
  // per-warp buffer of cbp float2: c_k for pass 1, then (general path) the window's values; pass 1
  // has read c before pass 2 writes the values, and the next image writes c after the loop's sync
  float2* cb = reinterpret_cast<float2*>(smem + a.off_s) + warp * a.cbp;
  float* sb = reinterpret_cast<float*>(cb);
  float* wlw = reinterpret_cast<float*>(smem + a.off_wl) + warp * a.sp;  // per warp [sp]

  // ---- shared tables
  {
    float4* x4w = reinterpret_cast<float4*>(smem + a.off_x);
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
    for (int i = tid; i < M / 2; i += NT) {
      const float4 v = __ldcg(xg + i);
      x4w[i] = v;
    }
    float2* tuw = reinterpret_cast<float2*>(smem + a.off_tu);
    for (int i = tid; i < KR * NUP; i += NT) tuw[i] = i < Kp1 * NUP ? a.tu[i] : make_float2(0.f, 0.f);
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    float* lrw = reinterpret_cast<float*>(smem + a.off_lr);
    for (int i = tid; i < Lw; i += NT) lrw[i] = __ldcg(a.logrho32 + i);
    int2* uw = reinterpret_cast<int2*>(smem + a.off_units);
    for (int i = tid; i < NUP; i += NT) uw[i] = a.units[i];
    float* wl0 = reinterpret_cast<float*>(smem + a.off_wl);
    for (int i = tid; i < a.sp * (NT / 32); i += NT) wl0[i] = 0.f;
    float2* cb0 = reinterpret_cast<float2*>(smem + a.off_s);
    for (int i = tid; i < a.cbp * (NT / 32); i += NT) cb0[i] = make_float2(0.f, 0.f);
    if (tid < 2 * nwarps) mbar_init(&bar[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();

  // ---- per-lane constants
  // pass 1: lane owns mirror unit u = lane (window indices ia and ib, ib absent: -inf)
  int ia = 0x3fffffff, ib = 0x3fffffff;
  float lra = -INFINITY, lrb = -INFINITY;
  if (lane < NU) {
    const int2 ab = uab[lane];
    ia = ab.x;
    lra = lrs[ab.x];
    if (ab.y >= 0) ib = ab.y, lrb = lrs[ab.y];
  }
  const float2* tcol = tus + min(lane, NUP - 1);
  // pass 2 and the back transform: lane j takes the distance d = j of its rows k = r + 8 m
  float2 tdr[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int k = r + 8 * m;
    tdr[m] = (k < Kp1 && j < a.nd) ? a.td[k * a.nd + j] : make_float2(0.f, 0.f);
  }

  const int gw = cta_ * nwarps + warp, GW = grid_ * nwarps;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  unsigned char* const wring = ring + (size_t)warp * 2 * a.slot_bytes;
  uint64_t* mybar = bar + 2 * warp;
  auto issue = [&](int im, int st) {
    if (im >= a.N) return;
    mbar_arrive_expect_tx(&mybar[st], img_bytes);
    bulk_g2s(wring + (size_t)st * a.slot_bytes, a.y + (size_t)im * M, img_bytes, &mybar[st]);
  };

  float4 acc[MR][QV];
#pragma unroll
  for (int m = 0; m < MR; ++m)
#pragma unroll
    for (int u = 0; u < QV; ++u) acc[m][u] = make_float4(0.f, 0.f, 0.f, 0.f);
  double ll_acc = 0.0, ysq_acc = 0.0;
  const float two_beta = a.two_beta;

  if (warp < nwarps && lane == 0) {
    issue(gw, 0);
    issue(gw + GW, 1);
  }
  auto load_shift = [&](int im) -> int {
    if (!a.shift || im >= a.N) return 0;
    int s = a.shift[im];
    if (s < 0 || s >= L) {
      s %= L;
      if (s < 0) s += L;
    }
    return s;
  };
  int sj_next = warp < nwarps ? load_shift(gw) : 0;

  for (int it = 0; warp < nwarps && gw + it * GW < a.N; ++it) {
    const int st = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const int img = gw + it * GW;
    const int sj = sj_next;
    sj_next = load_shift(img + GW);  // in flight while this image is processed
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

    // ---- correlation c_k = sum_q conj(y_kq) x_kq
    float2 c[MR];
    float2 sq = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int k = r + 8 * m;
      float2 P = make_float2(0.f, 0.f), Qv = make_float2(0.f, 0.f);
      if (m < MR - 1 || k < Kp1) {  // rows of all groups but the last exist
#pragma unroll
        for (int u = 0; u < QV; ++u) {
          const int pidx = k * row4 + j + 4 * u;
          const float4 yv = y4[pidx], xv = xs4[pidx];
          const float2 y01 = make_float2(yv.x, yv.y), y23 = make_float2(yv.z, yv.w);
          P = __ffma2_rn(y01, make_float2(xv.x, xv.y), P);
          P = __ffma2_rn(y23, make_float2(xv.z, xv.w), P);
          Qv = __ffma2_rn(y01, make_float2(xv.y, xv.x), Qv);
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
      c[m] = make_float2(cr, ci);
    }
    if (want_ysq) {
      const float t = warp_sum(sq.x + sq.y);
      if (lane == 0) ysq_acc += (double)t;
    }
    // ---- pass 1: lane-owned mirror units over all rows, c_k e^{-i k theta_hat_j} (the alignment)
    // broadcast from the per-warp buffer; the raw c stays in registers for pass 2
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const int k = r + 8 * m;
        if (m < MR - 1 || k < Kp1) cb[k] = c[m];
      }
    }
    __syncwarp();
    if (a.shift) {  // lane k rotates row k (and row k + 32)
#pragma unroll
      for (int k = lane; k < KR; k += 32) {
        if (k < Kp1) cb[k] = cmul(cb[k], tfs[mod_l(k * sj, L, invL)]);
      }
      __syncwarp();
    }
    float2 AB;
    {
      const float4* cb4 = reinterpret_cast<const float4*>(cb);  // rows >= K+1 are zero
      float2 ab[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) ab[t] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k2 = 0; k2 < KR / 2; ++k2) {
        const float4 cc = cb4[k2];  // rows 2 k2 and 2 k2 + 1
        ab[(2 * k2) & 3] = __ffma2_rn(make_float2(cc.x, cc.y), tcol[(2 * k2) * NUP], ab[(2 * k2) & 3]);
        ab[(2 * k2 + 1) & 3] = __ffma2_rn(make_float2(cc.z, cc.w), tcol[(2 * k2 + 1) * NUP], ab[(2 * k2 + 1) & 3]);
      }
      AB = __fadd2_rn(__fadd2_rn(ab[0], ab[1]), __fadd2_rn(ab[2], ab[3]));
    }
    const float sa1 = fmaf(two_beta, AB.x - AB.y, lra);  // offset +o (or the unit's only offset)
    const float sb1 = fmaf(two_beta, AB.x + AB.y, lrb);  // offset -o
    int peak, dist;
    float vref;
    {
      const float v = fmaxf(sa1, sb1);
      const int li = sa1 > sb1 ? ia : sb1 > sa1 ? ib : min(ia, ib);
      const int kmax = __reduce_max_sync(FULL, f2ord(v));
      int pk = __reduce_min_sync(FULL, f2ord(v) == kmax ? li : 0x7fffffff);
      if (pk >= Lw) pk = 0;  // only if every log-weight is -inf
      vref = ord2f(kmax);
      const float thr = vref - 40.f;
      int lo = pk, hi = pk;
      if (sa1 >= thr) lo = min(lo, ia), hi = max(hi, ia);
      if (sb1 >= thr) lo = min(lo, ib), hi = max(hi, ib);
      lo = __reduce_min_sync(FULL, lo);
      hi = __reduce_max_sync(FULL, hi);
      peak = pk;
      dist = max(pk - lo, hi - pk);
    }

    // ---- pass 2: c'_k = c_k e^{-i k (theta_hat_j + theta_l*)} (raw c, one rotation for the alignment and
    // the peak); S(l* +- d) - S(l*) = A_d -+ B_d with A_d = sum c'.x (cos t - 1), B_d = sum c'.y (-sin t),
    // t = 2 pi k d / L.  The same factors rotate W back below.
    const int p = peak, D = dist;
    int op = a.l0m + p + sj;
    if (op >= L) op -= L;
    if (op >= L) op -= L;
    float2 fk[MR], cq[MR];
    {
      int ph = mod_l(r * op, L, invL);
      const int pst = mod_l(8 * op, L, invL);
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        fk[m] = tfs[ph];
        cq[m] = cmul(c[m], fk[m]);
        ph += pst;
        if (ph >= L) ph -= L;
      }
    }
    const float lr_ref = lrs[p];
    float2 W[MR];
    if (D < 4) {
      // sharp image: lane j holds the distance d = j (summed over all rows below)
      float2 ad = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < MR; ++m) ad = __ffma2_rn(cq[m], tdr[m], ad);
      float da = ad.x - ad.y, db = ad.x + ad.y;
      da += __shfl_xor_sync(FULL, da, 4);
      db += __shfl_xor_sync(FULL, db, 4);
      da += __shfl_xor_sync(FULL, da, 8);
      db += __shfl_xor_sync(FULL, db, 8);
      da += __shfl_xor_sync(FULL, da, 16);
      db += __shfl_xor_sync(FULL, db, 16);
      const int la = p + j, lb = p - j;
      const bool va = j <= D && la < Lw, vb = j >= 1 && j <= D && lb >= 0;
      const float sa = va ? fmaf(two_beta, da, lrs[min(la, Lw - 1)] - lr_ref) : -INFINITY;
      const float sbv = vb ? fmaf(two_beta, db, lrs[max(lb, 0)] - lr_ref) : -INFINITY;
      float mx = fmaxf(sa, sbv);
      mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, 2));
      const float ea = __expf(sa - mx), eb = __expf(sbv - mx);
      float z = ea + eb;
      z += __shfl_xor_sync(FULL, z, 1);
      z += __shfl_xor_sync(FULL, z, 2);
      const float inv = 1.f / z;
      const float wa = ea * inv, wb = eb * inv;
      if (r == 0) {
        if (va) wlw[la] += wa;
        if (vb) wlw[lb] += wb;
      }
      if (lane == 0) ll_acc += (double)(vref + (mx + __logf(z)));
      if (a.w_out) {  // every lane runs the same trip count (the shuffles need the whole warp)
        float* wo = a.w_out + (size_t)img * Lw;
        for (int l0 = 0; l0 < Lw; l0 += 32) {
          const int l = l0 + lane, d = l - p;
          const float fa = __shfl_sync(FULL, wa, min(max(d, 0), 3));
          const float fb = __shfl_sync(FULL, wb, min(max(-d, 0), 3));
          if (l < Lw) wo[l] = (d >= 0 && d <= 3) ? fa : (d < 0 && d >= -3) ? fb : 0.f;
        }
      }
      // back transform around the peak: W_k e^{-i k theta_l*} = 1 + sum_{d>=1} [(w_{+d} + w_{-d}) (cos t - 1)
      //   + i (w_{-d} - w_{+d}) (-sin t)]
      const float2 swd = j >= 1 ? make_float2(wa + wb, wb - wa) : make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        float2 t = make_float2(swd.x * tdr[m].x, swd.y * tdr[m].y);
        t.x += __shfl_xor_sync(FULL, t.x, 1);
        t.y += __shfl_xor_sync(FULL, t.y, 1);
        t.x += __shfl_xor_sync(FULL, t.x, 2);
        t.y += __shfl_xor_sync(FULL, t.y, 2);
        W[m] = make_float2(1.f + t.x, t.y);
      }
    } else {
      // ---- general path (the warp sweep's): values within D of the peak into the per-warp buffer
      auto quad_sum = [&](float v) {
        v += __shfl_xor_sync(FULL, v, 4);
        v += __shfl_xor_sync(FULL, v, 8);
        v += __shfl_xor_sync(FULL, v, 16);
        return v;
      };
      const int nd1 = a.nd - 1;
      const float2* trow0 = a.td + r * a.nd;
      for (int d0 = 0; d0 <= D; d0 += 4 * kUnitChunk / 4) {
        constexpr int kT = kUnitChunk / 4;  // distance slots per lane per chunk
        const int nt = min(kT, (D - d0) / 4 + 1);
        float Ad[kT], Bd[kT];
#pragma unroll
        for (int t = 0; t < kT; ++t) Ad[t] = 0.f, Bd[t] = 0.f;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          if (m < MR - 1 || r + 8 * m < Kp1) {
            const float2* tr = trow0 + 8 * m * a.nd;
#pragma unroll
            for (int t = 0; t < kT; ++t) {
              if (t < nt) {
                const float2 tv = tr[min(d0 + j + 4 * t, nd1)];
                Ad[t] = fmaf(cq[m].x, tv.x, Ad[t]);
                Bd[t] = fmaf(cq[m].y, tv.y, Bd[t]);
              }
            }
          }
        }
#pragma unroll
        for (int t = 0; t < kT; ++t) {
          if (t < nt) {
            const int d = d0 + j + 4 * t;
            const float da = quad_sum(Ad[t] - Bd[t]), db = quad_sum(Ad[t] + Bd[t]);
            if (r == 0 && d <= D) {
              const int la = p + d, lb = p - d;
              if (la < Lw) sb[la] = fmaf(two_beta, da, lrs[la] - lr_ref);
              if (d > 0 && lb >= 0) sb[lb] = fmaf(two_beta, db, lrs[lb] - lr_ref);
            }
          }
        }
      }
      __syncwarp();
      auto near = [&](int l) { return l >= p - D && l <= p + D; };
      float mx = -INFINITY;
      for (int l = lane; l < Lw; l += 32)
        if (near(l)) mx = fmaxf(mx, sb[l]);
      mx = warp_max(mx);
      float z = 0.f;
      for (int l = lane; l < Lw; l += 32) {
        const float e = near(l) ? expf(sb[l] - mx) : 0.f;
        sb[l] = e;
        z += e;
      }
      z = warp_sum(z);
      const float inv = 1.f / z;
      float* wo = a.w_out ? a.w_out + (size_t)img * Lw : nullptr;
      for (int l = lane; l < Lw; l += 32) {
        const float w = sb[l] * inv;
        sb[l] = w;
        wlw[l] += w;
        if (wo) wo[l] = w;
      }
      if (lane == 0) ll_acc += (double)(vref + (mx + __logf(z)));
      __syncwarp();
      // back transform around the peak on the distance units d <= D
      auto wpair = [&](int d) {
        float wa = 0.f, wb = 0.f;
        if (d >= 1 && d <= D) {
          const int la = p + d, lb = p - d;
          if (la < Lw) wa = sb[la];
          if (lb >= 0) wb = sb[lb];
        }
        return make_float2(wa + wb, wb - wa);
      };
#pragma unroll
      for (int m = 0; m < MR; ++m) W[m] = make_float2(0.f, 0.f);
      for (int d0 = 0; d0 <= D; d0 += 4 * (kUnitChunk / 4)) {
        constexpr int kT = kUnitChunk / 4;
        const int nt = min(kT, (D - d0) / 4 + 1);
#pragma unroll
        for (int t = 0; t < kT; ++t) {
          if (t < nt) {
            const int d = d0 + j + 4 * t;
            const float2 sw = wpair(d);
#pragma unroll
            for (int m = 0; m < MR; ++m) {
              if (m < MR - 1 || r + 8 * m < Kp1) {
                const float2 tv = trow0[8 * m * a.nd + min(d, nd1)];
                W[m].x = fmaf(sw.x, tv.x, W[m].x);
                W[m].y = fmaf(sw.y, tv.y, W[m].y);
              }
            }
          }
        }
      }
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        W[m].x += __shfl_xor_sync(FULL, W[m].x, 1);
        W[m].y += __shfl_xor_sync(FULL, W[m].y, 1);
        W[m].x += __shfl_xor_sync(FULL, W[m].x, 2);
        W[m].y += __shfl_xor_sync(FULL, W[m].y, 2);
        W[m].x += 1.f;
      }
      __syncwarp();  // the next image rewrites sb only after every lane has read it
    }
    // one rotation by theta_hat_j + theta_l*, i.e. by (s_j + l0 + l*) mod L
#pragma unroll
    for (int m = 0; m < MR; ++m) W[m] = cmul_conj_b(W[m], fk[m]);

    // ---- accumulate W_k y_kq
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
    // ring stage st may be refilled once every lane has finished reading it (and cb is rewritten
    // by the next image only after every lane's pass 1 has read it)
    __syncwarp();
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(img + 2 * GW, st);
    }
  }

  // ---- CTA combination: per-warp FP32 sums through the (now idle) ring, then FP64 partials
  __syncthreads();
  if (tid < 2 * nwarps) mbar_inval(&bar[tid]);  // the CTA may run another sweep on this memory next
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
  const int G = a.G, cta = cta_;
  const float* redf = reinterpret_cast<const float*>(ring);
  for (int col = tid; col < 2 * M; col += NT) {
    float sum = 0.f;
    for (int w = 0; w < NT / 32; ++w) sum += redf[(size_t)w * 2 * M + col];
    a.part[(size_t)col * G + cta] = (double)sum;
  }
  for (int l = tid; l < Lw; l += NT) {
    float sum = 0.f;
    const float* wl0 = reinterpret_cast<const float*>(smem + a.off_wl);
    for (int w = 0; w < NT / 32; ++w) sum += wl0[w * a.sp + l];
    a.part[(size_t)(2 * M + l) * G + cta] = (double)sum;
  }
  __shared__ double red[2][32];
  if (lane == 0) red[0][warp] = ll_acc, red[1][warp] = ysq_acc;
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < NT / 32; ++w) t0 += red[0][w], t1 += red[1][w];
    a.part[(size_t)(2 * M + Lw) * G + cta] = t0;
    a.part[(size_t)(2 * M + Lw + 1) * G + cta] = t1;
  }
}

template <int QV, int MR, int NUPC>
__global__ void __launch_bounds__(SweepV5Shape<QV, MR>::kThreads, 1) k_sweep_v5(const SweepV2Args a) {
  sweep_v5_body<QV, MR, NUPC>(a, blockIdx.x, gridDim.x);
}

}  // namespace mra

// Instantiation table for one row width QV: MR = 1..7 rows per quad, unit pitch 20 or 40.
#define MRA_SWEEP_V5_CASE(QV, MR) \
  case MR: return nup == 20 ? SweepV2Launch{k_sweep_v5<QV, MR, 20>, SweepV5Shape<QV, MR>::kThreads} \
                            : SweepV2Launch{k_sweep_v5<QV, MR, 40>, SweepV5Shape<QV, MR>::kThreads};
#define MRA_SWEEP_V5_TABLE(QV)                     \
  namespace mra {                                  \
  SweepV2Launch sweep_v5_q##QV(int MR, int nup) {  \
    if (nup != 20 && nup != 40) return {nullptr, 0}; \
    switch (MR) {                                  \
      MRA_SWEEP_V5_CASE(QV, 1)                     \
      MRA_SWEEP_V5_CASE(QV, 2)                     \
      MRA_SWEEP_V5_CASE(QV, 3)                     \
      MRA_SWEEP_V5_CASE(QV, 4)                     \
      MRA_SWEEP_V5_CASE(QV, 5)                     \
      MRA_SWEEP_V5_CASE(QV, 6)                     \
      MRA_SWEEP_V5_CASE(QV, 7)                     \
      default: return {nullptr, 0};                \
    }                                              \
  }                                                \
  }
