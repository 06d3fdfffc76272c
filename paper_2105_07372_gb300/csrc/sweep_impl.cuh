// Warp-streaming EM sweep (rows of Q a multiple of 8 coefficients).
//
// Each warp owns a private shared-memory ring filled by bulk copies (one image
// per copy, IPW images per ring stage, two stages) and runs its images through
// every stage with warp-level synchronisation only.  The code is written for IPW
// images carried at once (the x and twiddle loads shared by them), but only
// IPW = 1 is built: two images per warp measured slower (fewer resident warps),
// and the peak-relative second pass and the wide-window paths handle one image.
//
//   lanes form 8 quads; quad r owns the rows k = r, r+8, r+16, ...; lane j of a
//   quad owns the float4 columns j, j+4, ... of those rows (QV of them per row).
//
//   correlation   c_k = sum_q conj(y_kq) x_kq        quad-local, two xor shuffles
//   forward       S_l = Re sum_k c_k e^{-i k theta_l}, window offsets grouped in
//                 mirror units {+o, -o}: A = sum c.x cos, B = sum c.y sin give
//                 S_{+o} = A - B and S_{-o} = A + B (halves the work)
//   normalise     w_l = exp(s_l - max) / Z over a per-warp buffer
//   back          W_k = sum_l w_l e^{+i k theta_l} = sum_units (w_+ + w_-) cos + i (w_- - w_+) sin
//   accumulate    num_kq += W_k y_kq into per-lane FP32 registers
//
// FP32 log-weights reach 2 beta S ~ thousands, and FP32 rounding of such sums (and of the
// twiddles) would move the normalised weights by more than 1e-5.  So pass 1 (above) only
// locates each image's peak rotation l* and how far from it the weights matter; pass 2
// recomputes those values as differences S(l* +- d) - S(l*) from c rotated to the peak and
// an FP64-built table of (cos t - 1, -sin t), whose terms vanish near the peak.
// Windows of one unit chunk hand each warp a fixed stride of images.  Wider windows cost per
// image in proportion to the spread of its posterior (pass 2 and the back transform run over
// the distances within D of the peak), so their warps take images one at a time from a counter
// in the control block once the first two (static) are done, and the last warp to finish
// clears the counter for the next launch.
// The CTA combines its warps' sums once at the end and writes FP64 partials.
#pragma once
#include "common.cuh"

namespace mra {

template <int QV, int MR, int IPW>
struct SweepV2Shape {
  static constexpr int kThreads = (IPW == 2 || MR * QV * 4 > 64) ? 256 : 512;
};

constexpr int kUC = 5;  // mirror units per lane per chunk

// a mod L for 0 <= a < 2^24 using a float reciprocal of L, corrected to the exact residue.
__device__ __forceinline__ int mod_small(int a, int L, float invL) {
  int m = a - __float2int_rz((float)a * invL) * L;
  if (m < 0) m += L;
  if (m >= L) m -= L;
  return m;
}

// LWC: lane-strided passes over the window (ceil(Lw / 32)) fixed at compile time (1 or 2) for a
// window of one unit chunk; 0 for any window; -1 for any window with the unit twiddle table read
// from global memory (windows whose table does not fit in shared memory next to the rings).
// The fixed counts let the per-image loops over the window and its units unroll (the unit
// table is then 4 kUC wide).
//
// The sweep is a device function of (arguments, CTA index, grid size), so that the batched
// persistent kernel can run it for one instance's CTA slot; k_sweep_v2 launches it directly.
template <int QV, int MR, int IPW, int LWC>
__device__ __forceinline__ void sweep_v2_body(const SweepV2Args& a, const int cta_, const int grid_) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = SweepV2Shape<QV, MR, IPW>::kThreads;
  // the state (x, log rho, control words) may come from another CTA of a persistent launch: read
  // it through L2
  if (__ldcg(&a.ctrl->done)) return;
  const bool want_ysq = (__ldcg(&a.ctrl->iter) == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = a.nwarps;  // <= NT/32 (warps beyond it only join the final combination)
  const int r = lane >> 2, j = lane & 3;
  const int Kp1 = a.Kp1, L = a.L, Lw = a.Lw, NU = a.NU, M = a.M;
  const bool wrap = a.wrap != 0;
  const int NUP = LWC > 0 ? 4 * kUC : a.NUP;
  // f(l) for this lane's window indices l = lane, lane + 32, ...
  auto for_window = [&](auto&& f) {
    if constexpr (LWC > 0) {
#pragma unroll
      for (int t = 0; t < LWC; ++t) {
        const int l = lane + 32 * t;
        if (l < Lw) f(l);
      }
    } else {
      for (int l = lane; l < Lw; l += 32) f(l);
    }
  };
  const float invL = 1.0f / (float)L;
  constexpr int row4 = QV * 4;  // float4 per row

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);  // [NT/32][2]
  unsigned char* ring = smem + a.off_ring;            // [nwarps][2][IPW][slot]
  const float4* xs4 = reinterpret_cast<const float4*>(smem + a.off_x);
  const float2* tus = LWC >= 0 ? reinterpret_cast<const float2*>(smem + a.off_tu) : a.tu;  // [Kp1][NUP]
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);  // [L]
  const float* lrs = reinterpret_cast<const float*>(smem + a.off_lr);    // [Lw]
  const int2* uab = reinterpret_cast<const int2*>(smem + a.off_units);   // [NUP] (a, b) window indices, b < 0: single
  float* sbuf0 = reinterpret_cast<float*>(smem + a.off_s) + warp * IPW * a.sp;  // per warp [IPW][sp]
  float* wlw = reinterpret_cast<float*>(smem + a.off_wl) + warp * a.sp;          // per warp [sp]

  // ---- shared tables
  {
    float4* x4w = reinterpret_cast<float4*>(smem + a.off_x);
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
    for (int i = tid; i < M / 2; i += NT) x4w[i] = __ldcg(xg + i);
    if constexpr (LWC >= 0) {
      float2* tuw = reinterpret_cast<float2*>(smem + a.off_tu);
      for (int i = tid; i < Kp1 * NUP; i += NT) tuw[i] = a.tu[i];
    }
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    float* lrw = reinterpret_cast<float*>(smem + a.off_lr);
    for (int i = tid; i < Lw; i += NT) lrw[i] = __ldcg(a.logrho32 + i);
    int2* uw = reinterpret_cast<int2*>(smem + a.off_units);
    for (int i = tid; i < NUP; i += NT) uw[i] = a.units[i];
    float* wl0 = reinterpret_cast<float*>(smem + a.off_wl);
    for (int i = tid; i < a.sp * (NT / 32); i += NT) wl0[i] = 0.f;
    if (tid < 2 * nwarps) mbar_init(&bar[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();

  const int gw = cta_ * nwarps + warp, GW = grid_ * nwarps;
  constexpr bool kDyn = LWC <= 0 && IPW == 1;  // images handed out one at a time
  int held0 = gw, held1 = gw + GW;              // kDyn: the image in ring stage 0 / 1 (>= N: none)
  const uint32_t img_bytes = (uint32_t)M * 8u;
  unsigned char* const wring = ring + (size_t)warp * 2 * IPW * a.slot_bytes;
  uint64_t* mybar = bar + 2 * warp;
  // ring stage st (0/1) holds group p's images; image i of it sits in slot st * IPW + i
  auto issue = [&](int p, int st) {
    int nv = 0;
#pragma unroll
    for (int i = 0; i < IPW; ++i) nv += (gw + (p * IPW + i) * GW < a.N) ? 1 : 0;
    if (nv == 0) return;
    mbar_arrive_expect_tx(&mybar[st], (uint32_t)nv * img_bytes);
#pragma unroll
    for (int i = 0; i < IPW; ++i) {
      const int im = gw + (p * IPW + i) * GW;
      if (im < a.N)
        bulk_g2s(wring + (size_t)(st * IPW + i) * a.slot_bytes, a.y + (size_t)im * M, img_bytes, &mybar[st]);
    }
  };

  float4 acc[MR][QV];
#pragma unroll
  for (int m = 0; m < MR; ++m)
#pragma unroll
    for (int u = 0; u < QV; ++u) acc[m][u] = make_float4(0.f, 0.f, 0.f, 0.f);
  double ll_acc = 0.0, ysq_acc = 0.0;
  const float two_beta = a.two_beta;

  if (warp < nwarps && lane == 0) {
    issue(0, 0);
    issue(1, 1);
  }

  for (int p = 0; warp < nwarps && (kDyn ? ((p & 1) ? held1 : held0) : gw + p * IPW * GW) < a.N; ++p) {
    const int st = p & 1;
    const uint32_t parity = (uint32_t)((p >> 1) & 1);
    const bool ok = mbar_wait_bounded(&mybar[st], parity);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        mbar_wait_bounded(&mybar[st], parity);
        if ((kDyn ? (st ? held0 : held1) : gw + (p + 1) * IPW * GW) < a.N)
          mbar_wait_bounded(&mybar[st ^ 1], (uint32_t)(((p + 1) >> 1) & 1));
      }
      break;
    }
    int img[IPW];
    bool valid[IPW];
    const float4* y4[IPW];
    int ph0[IPW], phstep[IPW], sjv[IPW];
#pragma unroll
    for (int i = 0; i < IPW; ++i) {
      img[i] = kDyn ? (st ? held1 : held0) : gw + (p * IPW + i) * GW;
      valid[i] = img[i] < a.N;
      y4[i] = reinterpret_cast<const float4*>(wring + (size_t)(st * IPW + i) * a.slot_bytes);
      int sj = 0;
      if (a.shift && valid[i]) {
        sj = a.shift[img[i]] % L;
        if (sj < 0) sj += L;
      }
      sjv[i] = sj;
      ph0[i] = mod_small(r * sj, L, invL);
      phstep[i] = mod_small(8 * sj, L, invL);
    }

    float2 W[IPW][MR];
    if (a.align_only) {
      // weights are exactly 1 at offset 0: W_k = e^{+i k theta_hat_j}
#pragma unroll
      for (int i = 0; i < IPW; ++i) {
        int ph = ph0[i];
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          const float2 t = tfs[ph];
          W[i][m] = make_float2(t.x, -t.y);
          ph += phstep[i];
          if (ph >= L) ph -= L;
        }
      }
    } else {
      // ---- correlation (x loads shared by the IPW images)
      float2 c[IPW][MR];
      float sq[IPW];
#pragma unroll
      for (int i = 0; i < IPW; ++i) sq[i] = 0.f;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const int k = r + 8 * m;
        float cr[IPW], ci[IPW];
#pragma unroll
        for (int i = 0; i < IPW; ++i) cr[i] = 0.f, ci[i] = 0.f;
        if (m < MR - 1 || k < Kp1) {  // rows of all groups but the last exist
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const int pidx = k * row4 + j + 4 * u;
            const float4 xv = xs4[pidx];
#pragma unroll
            for (int i = 0; i < IPW; ++i) {
              const float4 yv = y4[i][pidx];
              cr[i] = fmaf(yv.x, xv.x, cr[i]); cr[i] = fmaf(yv.y, xv.y, cr[i]);
              ci[i] = fmaf(yv.x, xv.y, ci[i]); ci[i] = fmaf(-yv.y, xv.x, ci[i]);
              cr[i] = fmaf(yv.z, xv.z, cr[i]); cr[i] = fmaf(yv.w, xv.w, cr[i]);
              ci[i] = fmaf(yv.z, xv.w, ci[i]); ci[i] = fmaf(-yv.w, xv.z, ci[i]);
              if (want_ysq) {
                sq[i] = fmaf(yv.x, yv.x, sq[i]); sq[i] = fmaf(yv.y, yv.y, sq[i]);
                sq[i] = fmaf(yv.z, yv.z, sq[i]); sq[i] = fmaf(yv.w, yv.w, sq[i]);
              }
            }
          }
        }
#pragma unroll
        for (int i = 0; i < IPW; ++i) {
          cr[i] += __shfl_xor_sync(0xffffffffu, cr[i], 1);
          ci[i] += __shfl_xor_sync(0xffffffffu, ci[i], 1);
          cr[i] += __shfl_xor_sync(0xffffffffu, cr[i], 2);
          ci[i] += __shfl_xor_sync(0xffffffffu, ci[i], 2);
          c[i][m] = make_float2(cr[i], ci[i]);
        }
      }
      if (want_ysq) {
#pragma unroll
        for (int i = 0; i < IPW; ++i) {
          const float t = warp_sum(sq[i]);
          if (lane == 0 && valid[i]) ysq_acc += (double)t;
        }
      }
      if (a.shift) {  // c_k e^{-i k theta_hat_j}
#pragma unroll
        for (int i = 0; i < IPW; ++i) {
          int ph = ph0[i];
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            c[i][m] = cmul(c[i][m], tfs[ph]);
            ph += phstep[i];
            if (ph >= L) ph -= L;
          }
        }
      }

      // ---- forward transform, pass 1 over mirror units (chunks of 4 * kUC units): the peak l* and
      // the distance D from it beyond which every value is more than 40 below the peak's
      auto quad_sum = [&](float v) {
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        return v;
      };
      // per-quad partials of this lane's units for all IPW images (twiddle loads shared)
      auto partials = [&](int u0, float (&A)[IPW][kUC], float (&Bv)[IPW][kUC]) {
#pragma unroll
        for (int i = 0; i < IPW; ++i)
#pragma unroll
          for (int t = 0; t < kUC; ++t) A[i][t] = 0.f, Bv[i][t] = 0.f;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          const int k = r + 8 * m;
          if (m < MR - 1 || k < Kp1) {  // rows of all groups but the last exist
            const float2* trow = tus + k * NUP + u0 + j;
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              const float2 tv = trow[4 * t];
#pragma unroll
              for (int i = 0; i < IPW; ++i) {
                A[i][t] = fmaf(c[i][m].x, tv.x, A[i][t]);
                Bv[i][t] = fmaf(c[i][m].y, tv.y, Bv[i][t]);
              }
            }
          }
        }
      };
      // D from the lowest and highest window index whose value is within 40 of the peak (the
      // whole half circle when the window is all of it)
      auto peak_dist = [&](int p, int lo, int hi) {
        if (wrap) return L / 2;
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        return max(p - lo, hi - p);
      };
      float vref[IPW];  // FP32 log-weight at the peak l* (absolute)
      int peak[IPW], dist[IPW];
      if (NUP == 4 * kUC) {
        float A[IPW][kUC], Bv[IPW][kUC];
        partials(0, A, Bv);
#pragma unroll
        for (int i = 0; i < IPW; ++i) {
          float sa[kUC], sm[kUC];  // values at each unit's first offset and at its mirror
          int2 abt[kUC];
          float bv = -INFINITY;
          int bl = 0x7fffffff;
#pragma unroll
          for (int t = 0; t < kUC; ++t) {
            const int u = j + 4 * t;
            const float At = quad_sum(A[i][t]), Bt = quad_sum(Bv[i][t]);
            sa[t] = -INFINITY, sm[t] = -INFINITY;
            abt[t] = make_int2(0, 0);
            if (u < NU) {
              const int2 ab = uab[u];
              abt[t] = ab;
              sa[t] = fmaf(two_beta, At - Bt, lrs[ab.x]);
              if (sa[t] > bv || (sa[t] == bv && ab.x < bl)) bv = sa[t], bl = ab.x;
              if (ab.y >= 0) {
                sm[t] = fmaf(two_beta, At + Bt, lrs[ab.y]);
                if (sm[t] > bv || (sm[t] == bv && ab.y < bl)) bv = sm[t], bl = ab.y;
              }
            }
          }
#pragma unroll
          for (int o = 1; o <= 2; o <<= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (ov > bv || (ov == bv && ol < bl)) bv = ov, bl = ol;
          }
          if (bl >= Lw) bl = 0;  // only if every log-weight is -inf
          vref[i] = bv;
          peak[i] = bl;
          const float thr = bv - 40.f;
          int lo = bl, hi = bl;
#pragma unroll
          for (int t = 0; t < kUC; ++t) {  // sa, sm are -inf where a unit or its mirror is absent
            if (sa[t] >= thr) lo = min(lo, abt[t].x), hi = max(hi, abt[t].x);
            if (sm[t] >= thr) lo = min(lo, abt[t].y), hi = max(hi, abt[t].y);
          }
          dist[i] = peak_dist(bl, lo, hi);
        }
      } else if constexpr (IPW == 1) {
        // wide windows: each lane owns whole units (u0 + lane, u0 + lane + 32) and sums over every row,
        // with c_k broadcast from its quad (row k sits in quad k mod 8 as c[k / 8]) and coalesced
        // twiddle rows, so no cross-lane reduction is needed per unit
        float* sb = sbuf0;
        for (int u0 = 0; u0 < NU; u0 += 64) {  // pass 1 into the per-warp buffer
          const int ua = u0 + lane, ub = ua + 32;
          const float2* ta = tus + min(ua, NUP - 1);
          const float2* tb = tus + min(ub, NUP - 1);
          float A0 = 0.f, B0 = 0.f, A1 = 0.f, B1 = 0.f;
#pragma unroll
          for (int k = 0; k < 8 * MR; ++k) {
            if (k < 8 * (MR - 1) || k < Kp1) {  // static for all row groups but the last: loads batch
              const float cx = __shfl_sync(0xffffffffu, c[0][k >> 3].x, 4 * (k & 7));
              const float cy = __shfl_sync(0xffffffffu, c[0][k >> 3].y, 4 * (k & 7));
              const float2 va = ta[k * NUP], vb = tb[k * NUP];
              A0 = fmaf(cx, va.x, A0); B0 = fmaf(cy, va.y, B0);
              A1 = fmaf(cx, vb.x, A1); B1 = fmaf(cy, vb.y, B1);
            }
          }
          if (ua < NU) {
            const int2 ab = uab[ua];
            sb[ab.x] = fmaf(two_beta, A0 - B0, lrs[ab.x]);
            if (ab.y >= 0) sb[ab.y] = fmaf(two_beta, A0 + B0, lrs[ab.y]);
          }
          if (ub < NU) {
            const int2 ab = uab[ub];
            sb[ab.x] = fmaf(two_beta, A1 - B1, lrs[ab.x]);
            if (ab.y >= 0) sb[ab.y] = fmaf(two_beta, A1 + B1, lrs[ab.y]);
          }
        }
        __syncwarp();
        float bv = -INFINITY;
        int bl = 0x7fffffff;
        for_window([&](int l) {
          const float v = sb[l];
          if (v > bv) bv = v, bl = l;
        });
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
          if (ov > bv || (ov == bv && ol < bl)) bv = ov, bl = ol;
        }
        if (bl >= Lw) bl = 0;
        vref[0] = bv;
        peak[0] = bl;
        const float thr = bv - 40.f;
        int lo = bl, hi = bl;
        for_window([&](int l) {
          if (sb[l] >= thr) lo = min(lo, l), hi = max(hi, l);
        });
        dist[0] = peak_dist(bl, lo, hi);
        __syncwarp();  // pass 2 rewrites sb
      }

      // ---- pass 2: the values within D of the peak, relative to it, from c rotated to the peak,
      // c'_k = c_k e^{-i k theta_l*}, and the distance-unit table (cos t - 1, -sin t),
      // t = 2 pi k d step / L: S(l* + d) - S(l*) = A_d - B_d and S(l* - d) - S(l*) = A_d + B_d with
      // A_d = sum c'.x (cos t - 1), B_d = sum c'.y (-sin t).  The terms are small near the peak,
      // so the FP32 differences keep their precision however large 2 beta |c| is.  Values
      // farther than D are more than 40 below the peak: their weights (< e^-40) are taken as 0.
#pragma unroll
      for (int i = 0; i < IPW; ++i) {
        const int p = peak[i], D = dist[i];
        float2 cq[MR];
        if (a.tw) {  // dense window: the window twiddle table (global, L1-resident)
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            const int k = r + 8 * m;
            cq[m] = (m < MR - 1 || k < Kp1) ? cmul(c[i][m], a.tw[k * a.twp + p]) : make_float2(0.f, 0.f);
          }
        } else {
          int op = a.l0m + p;
          if (op >= L) op -= L;
          int ph = mod_small(r * op, L, invL);
          const int pst = mod_small(8 * op, L, invL);
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            cq[m] = cmul(c[i][m], tfs[ph]);
            ph += pst;
            if (ph >= L) ph -= L;
          }
        }
        float* sb = sbuf0 + i * a.sp;
        const float lr_ref = lrs[p];
        // one slot per lane and distance chunk: d = d0 + j (+ 4 t), four distances per quad
        auto emit = [&](int d, float Ad, float Bd) {
          const float da = quad_sum(Ad - Bd), db = quad_sum(Ad + Bd);
          if (r == 0 && d <= D) {
            int la = p + d, lb = p - d;
            if (wrap) {
              if (la >= L) la -= L;
              if (lb < 0) lb += L;
            }
            if (wrap || la < Lw) sb[la] = fmaf(two_beta, da, lrs[la] - lr_ref);
            if (d > 0 && (wrap ? 2 * d != L : lb >= 0)) sb[lb] = fmaf(two_beta, db, lrs[lb] - lr_ref);
          }
        };
        const int nd1 = a.nd - 1;
        const float2* trow0 = a.td + r * a.nd;  // row k = r; row r + 8 m is 8 m nd further
        if (D < 4) {  // the usual case: one distance per lane
          const float2* tp = trow0 + min(j, nd1);
          float Ad = 0.f, Bd = 0.f;
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            if (m < MR - 1 || r + 8 * m < Kp1) {
              const float2 tv = tp[8 * m * a.nd];
              Ad = fmaf(cq[m].x, tv.x, Ad);
              Bd = fmaf(cq[m].y, tv.y, Bd);
            }
          }
          emit(j, Ad, Bd);
        } else if constexpr (LWC <= 0) {
          // wide windows: lanes own whole distances (d0 + lane, d0 + lane + 32), c' broadcast by row
          // as in pass 1
          auto emit_lane = [&](int d, float Ad, float Bd) {
            if (d <= D) {
              int la = p + d, lb = p - d;
              if (wrap) {
                if (la >= L) la -= L;
                if (lb < 0) lb += L;
              }
              if (wrap || la < Lw) sb[la] = fmaf(two_beta, Ad - Bd, lrs[la] - lr_ref);
              if (d > 0 && (wrap ? 2 * d != L : lb >= 0)) sb[lb] = fmaf(two_beta, Ad + Bd, lrs[lb] - lr_ref);
            }
          };
          for (int d0 = 0; d0 <= D; d0 += 64) {
            const int da = d0 + lane, db = da + 32;
            const float2* ta = a.td + min(da, nd1);
            const float2* tb = a.td + min(db, nd1);
            float A0 = 0.f, B0 = 0.f, A1 = 0.f, B1 = 0.f;
#pragma unroll
            for (int k = 0; k < 8 * MR; ++k) {
              if (k < 8 * (MR - 1) || k < Kp1) {
                const float cx = __shfl_sync(0xffffffffu, cq[k >> 3].x, 4 * (k & 7));
                const float cy = __shfl_sync(0xffffffffu, cq[k >> 3].y, 4 * (k & 7));
                const float2 va = ta[k * a.nd], vb = tb[k * a.nd];
                A0 = fmaf(cx, va.x, A0); B0 = fmaf(cy, va.y, B0);
                A1 = fmaf(cx, vb.x, A1); B1 = fmaf(cy, vb.y, B1);
              }
            }
            emit_lane(da, A0, B0);
            emit_lane(db, A1, B1);
          }
        } else {
          for (int d0 = 0; d0 <= D; d0 += 4 * kUC) {
            const int nt = min(kUC, (D - d0) / 4 + 1);  // slots t holding some d <= D
            float Ad[kUC], Bd[kUC];
#pragma unroll
            for (int t = 0; t < kUC; ++t) Ad[t] = 0.f, Bd[t] = 0.f;
#pragma unroll
            for (int m = 0; m < MR; ++m) {
              if (m < MR - 1 || r + 8 * m < Kp1) {
                const float2* tr = trow0 + 8 * m * a.nd;
#pragma unroll
                for (int t = 0; t < kUC; ++t) {
                  if (t < nt) {
                    const float2 tv = tr[min(d0 + j + 4 * t, nd1)];
                    Ad[t] = fmaf(cq[m].x, tv.x, Ad[t]);
                    Bd[t] = fmaf(cq[m].y, tv.y, Bd[t]);
                  }
                }
              }
            }
#pragma unroll
            for (int t = 0; t < kUC; ++t)
              if (t < nt) emit(d0 + j + 4 * t, Ad[t], Bd[t]);
          }
        }
      }
      __syncwarp();

      // ---- normalisation over the window (values within D of the peak, relative to it; 0 beyond)
#pragma unroll
      for (int i = 0; i < IPW; ++i) {
        float* sb = sbuf0 + i * a.sp;
        const int p = peak[i], D = dist[i];
        auto near = [&](int l) { return wrap || (l >= p - D && l <= p + D); };
        float mx = -INFINITY;
        for_window([&](int l) {
          if (near(l)) mx = fmaxf(mx, sb[l]);
        });
        mx = warp_max(mx);
        float z = 0.f;
        for_window([&](int l) {
          const float e = near(l) ? expf(sb[l] - mx) : 0.f;
          sb[l] = e;
          z += e;
        });
        z = warp_sum(z);
        const float inv = 1.f / z;
        float* wo = (a.w_out && valid[i]) ? a.w_out + (size_t)img[i] * Lw : nullptr;
        for_window([&](int l) {
          const float w = sb[l] * inv;
          sb[l] = w;
          if (valid[i]) wlw[l] += w;
          if (wo) wo[l] = w;
        });
        // one FP64 add per image (FP64 instructions are costly here); the FP32 term is exact to ~1e-7
        if (lane == 0 && valid[i]) ll_acc += (double)(vref[i] + (mx + __logf(z)));
      }
      __syncwarp();

      if constexpr (LWC > 0) {
      // ---- back transform of a one-chunk window over its units (shared-memory twiddles, loads shared by
      // the IPW images); wider windows use the distance units around the peak (below)
#pragma unroll
      for (int i = 0; i < IPW; ++i)
#pragma unroll
        for (int m = 0; m < MR; ++m) W[i][m] = make_float2(0.f, 0.f);
      for (int u0 = 0; u0 < NUP; u0 += 4 * kUC) {
        float sw[IPW][kUC], dw[IPW][kUC];
#pragma unroll
        for (int t = 0; t < kUC; ++t) {
          const int u = u0 + j + 4 * t;
          int2 ab = make_int2(0, -1);
          if (u < NU) ab = uab[u];
#pragma unroll
          for (int i = 0; i < IPW; ++i) {
            const float* sb = sbuf0 + i * a.sp;
            const float wa = u < NU ? sb[ab.x] : 0.f;
            const float wb = (u < NU && ab.y >= 0) ? sb[ab.y] : 0.f;
            sw[i][t] = wa + wb;
            dw[i][t] = wb - wa;
          }
        }
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          const int k = r + 8 * m;
          if (m < MR - 1 || k < Kp1) {  // rows of all groups but the last exist
            const float2* trow = tus + k * NUP + u0 + j;
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              const float2 tv = trow[4 * t];
#pragma unroll
              for (int i = 0; i < IPW; ++i) {
                W[i][m].x = fmaf(sw[i][t], tv.x, W[i][m].x);
                W[i][m].y = fmaf(dw[i][t], tv.y, W[i][m].y);
              }
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < IPW; ++i) {
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          W[i][m].x += __shfl_xor_sync(0xffffffffu, W[i][m].x, 1);
          W[i][m].y += __shfl_xor_sync(0xffffffffu, W[i][m].y, 1);
          W[i][m].x += __shfl_xor_sync(0xffffffffu, W[i][m].x, 2);
          W[i][m].y += __shfl_xor_sync(0xffffffffu, W[i][m].y, 2);
        }
        if (a.shift) {  // W_k e^{+i k theta_hat_j}
          int ph = ph0[i];
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            W[i][m] = cmul_conj_b(W[i][m], tfs[ph]);
            ph += phstep[i];
            if (ph >= L) ph -= L;
          }
        }
      }
      } else {
      // ---- back transform around the peak, on the distance units as in pass 2:
      // W_k = e^{+i k (theta_hat_j + theta_l*)} (1 + sum_{d>=1} [(w_{l*+d} + w_{l*-d}) (cos t - 1)
      //        + i (w_{l*-d} - w_{l*+d}) (-sin t)]),  t = 2 pi k d step / L  (sum_l w_l = 1),
      // over d <= D only (weights beyond D are zero): one distance per lane in the usual D < 4.
#pragma unroll
      for (int i = 0; i < IPW; ++i) {
        const int p = peak[i], D = dist[i];
        const float* sb = sbuf0 + i * a.sp;
        auto wpair = [&](int d) {  // (w_{p+d} + w_{p-d}, w_{p-d} - w_{p+d}) for 1 <= d <= D
          float wa = 0.f, wb = 0.f;
          if (d >= 1 && d <= D) {
            int la = p + d, lb = p - d;
            if (wrap) {
              if (la >= L) la -= L;
              if (lb < 0) lb += L;
              wa = sb[la];
              if (2 * d != L) wb = sb[lb];
            } else {
              if (la < Lw) wa = sb[la];
              if (lb >= 0) wb = sb[lb];
            }
          }
          return make_float2(wa + wb, wb - wa);
        };
#pragma unroll
        for (int m = 0; m < MR; ++m) W[i][m] = make_float2(0.f, 0.f);
        const int nd1 = a.nd - 1;
        const float2* trow0 = a.td + r * a.nd;  // row k = r; row r + 8 m is 8 m nd further
        if (D < 4) {
          const float2 sw = wpair(j);
          const float2* tp = trow0 + min(j, nd1);
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            if (m < MR - 1 || r + 8 * m < Kp1) {
              const float2 tv = tp[8 * m * a.nd];
              W[i][m].x = fmaf(sw.x, tv.x, W[i][m].x);
              W[i][m].y = fmaf(sw.y, tv.y, W[i][m].y);
            }
          }
        } else {
          for (int d0 = 0; d0 <= D; d0 += 4 * kUC) {
            const int nt = min(kUC, (D - d0) / 4 + 1);
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              if (t < nt) {
                const int d = d0 + j + 4 * t;
                const float2 sw = wpair(d);
#pragma unroll
                for (int m = 0; m < MR; ++m) {
                  if (m < MR - 1 || r + 8 * m < Kp1) {
                    const float2 tv = trow0[8 * m * a.nd + min(d, nd1)];
                    W[i][m].x = fmaf(sw.x, tv.x, W[i][m].x);
                    W[i][m].y = fmaf(sw.y, tv.y, W[i][m].y);
                  }
                }
              }
            }
          }
        }
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          W[i][m].x += __shfl_xor_sync(0xffffffffu, W[i][m].x, 1);
          W[i][m].y += __shfl_xor_sync(0xffffffffu, W[i][m].y, 1);
          W[i][m].x += __shfl_xor_sync(0xffffffffu, W[i][m].x, 2);
          W[i][m].y += __shfl_xor_sync(0xffffffffu, W[i][m].y, 2);
          W[i][m].x += 1.f;
        }
        if (a.tw) {  // dense window: the peak's angle from the window table, then the shift
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            const int k = r + 8 * m;
            if (m < MR - 1 || k < Kp1) W[i][m] = cmul_conj_b(W[i][m], a.tw[k * a.twp + p]);
          }
          if (a.shift) {
            int ph = ph0[i];
#pragma unroll
            for (int m = 0; m < MR; ++m) {
              W[i][m] = cmul_conj_b(W[i][m], tfs[ph]);
              ph += phstep[i];
              if (ph >= L) ph -= L;
            }
          }
        } else {  // grid: one rotation by theta_hat_j + theta_l*, i.e. by (s_j + l0 + l*) mod L
          int op = a.l0m + p;
          if (op >= L) op -= L;
          int q = sjv[i] + op;
          if (q >= L) q -= L;
          int ph = mod_small(r * q, L, invL);
          const int pst = mod_small(8 * q, L, invL);
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            W[i][m] = cmul_conj_b(W[i][m], tfs[ph]);
            ph += pst;
            if (ph >= L) ph -= L;
          }
        }
      }
      }
    }

    // ---- accumulate W_k y_kq
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int k = r + 8 * m;
      if (m < MR - 1 || k < Kp1) {  // rows of all groups but the last exist
#pragma unroll
        for (int i = 0; i < IPW; ++i) {
          if (!valid[i]) continue;
          const float2 w = W[i][m];
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const float4 yv = y4[i][k * row4 + j + 4 * u];
            float4& q = acc[m][u];
            q.x = fmaf(w.x, yv.x, q.x); q.x = fmaf(-w.y, yv.y, q.x);
            q.y = fmaf(w.x, yv.y, q.y); q.y = fmaf(w.y, yv.x, q.y);
            q.z = fmaf(w.x, yv.z, q.z); q.z = fmaf(-w.y, yv.w, q.z);
            q.w = fmaf(w.x, yv.w, q.w); q.w = fmaf(w.y, yv.z, q.w);
          }
        }
      }
    }
    // ring stage st may be refilled once every lane has finished reading it
    __syncwarp();
    if constexpr (kDyn) {
      int nxt = 0;
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        nxt = 2 * GW + (int)atomicAdd(&a.ctrl->sched[0], 1u);
        if (nxt < a.N) {
          mbar_arrive_expect_tx(&mybar[st], img_bytes);
          bulk_g2s(wring + (size_t)st * a.slot_bytes, a.y + (size_t)nxt * M, img_bytes, &mybar[st]);
        }
      }
      nxt = __shfl_sync(0xffffffffu, nxt, 0);
      if (st) held1 = nxt;
      else held0 = nxt;
    } else if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(p + 2, st);
    }
  }
  if constexpr (kDyn) {  // the last warp out clears the counters (every fetch of this launch is done)
    if (warp < nwarps && lane == 0 &&
        atomicAdd(&a.ctrl->sched[1], 1u) == (unsigned)(grid_ * nwarps) - 1u) {
      atomicExch(&a.ctrl->sched[0], 0u);
      atomicExch(&a.ctrl->sched[1], 0u);
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
    if (m < MR - 1 || k < Kp1) {  // rows of all groups but the last exist
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

template <int QV, int MR, int IPW, int LWC>
__global__ void __launch_bounds__(SweepV2Shape<QV, MR, IPW>::kThreads, 1) k_sweep_v2(const SweepV2Args a) {
  sweep_v2_body<QV, MR, IPW, LWC>(a, blockIdx.x, gridDim.x);
}

}  // namespace mra

// Instantiation table for one row width QV: MR = 1..7 rows per quad, one image per warp
// (two images per warp measured slower and are not built), window passes lwc = 1, 2 or any (0;
// -1 with the unit table in global memory).
#define MRA_SWEEP_V2_CASE(QV, MR)                                                                       \
  case MR:                                                                                              \
    if (ipw != 1) return SweepV2Launch{nullptr, 0};                                                     \
    return lwc == 1  ? SweepV2Launch{k_sweep_v2<QV, MR, 1, 1>, SweepV2Shape<QV, MR, 1>::kThreads}       \
         : lwc == 2  ? SweepV2Launch{k_sweep_v2<QV, MR, 1, 2>, SweepV2Shape<QV, MR, 1>::kThreads}       \
         : lwc == -1 ? SweepV2Launch{k_sweep_v2<QV, MR, 1, -1>, SweepV2Shape<QV, MR, 1>::kThreads}      \
                     : SweepV2Launch{k_sweep_v2<QV, MR, 1, 0>, SweepV2Shape<QV, MR, 1>::kThreads};
#define MRA_SWEEP_V2_TABLE(QV)                              \
  namespace mra {                                          \
  SweepV2Launch sweep_v2_q##QV(int MR, int ipw, int lwc) { \
    switch (MR) {                                          \
      MRA_SWEEP_V2_CASE(QV, 1)                             \
      MRA_SWEEP_V2_CASE(QV, 2)                             \
      MRA_SWEEP_V2_CASE(QV, 3)                             \
      MRA_SWEEP_V2_CASE(QV, 4)                             \
      MRA_SWEEP_V2_CASE(QV, 5)                             \
      MRA_SWEEP_V2_CASE(QV, 6)                             \
      MRA_SWEEP_V2_CASE(QV, 7)                             \
      default: return {nullptr, 0};                        \
    }                                                      \
  }                                                        \
  }
