// Paired-warp EM sweep for grid windows of at most 32 mirror units (rows of Q a multiple of 8
// coefficients), Eq. weights_2d_em and Eq. coefficients_update.
//
// Two warps share each image.  Warp h of a pair owns the rows k = 1 + 8 MR h + 8 m + r
// (quad r = lane / 4, m < MR), lane j = lane % 4 of a quad the float4 columns j, j + 4, ...;
// so y, x and the accumulators of a lane are MR x QV float4 each and all stay in registers:
// y is read from shared memory once per image, x never.  The k = 0 row needs no transform: its
// twiddle is 1 for every rotation, so it adds the same amount to every log-weight (it cancels in
// the posterior) and W_0 = sum_l w_l = 1.  Warp 0 therefore only adds y_0q to its accumulators;
// the likelihood's k = 0 term, summed over the images of a CTA, is 2 beta Re <sum_j y_j0, x_0>,
// added once at the end.
//
//   correlation   c_k = sum_q conj(y_kq) x_kq over each warp's rows, reduced within quads
//   pass 1        each lane owns one mirror unit {+o, -o}; a warp's partial over its rows from
//                 c_k (shared-memory broadcast) and the unit table (two rows per 16-byte load);
//                 the two partials meet in shared memory at the first pair barrier, and both
//                 warps add them in the same order, so they take identical decisions: the peak
//                 l* and the distance D holding every log-weight within 40 of it
//   pass 2        c rotated to the peak (one rotation for the alignment and the peak), the
//                 FP64-built (cos t - 1, -sin t) table: exact differences from the peak, partial
//                 per warp, combined at the second pair barrier
//   sharp images  (D < 4, the usual case) normalised in registers and back-transformed over the
//                 distances in the "1 + sum" form; others through per-warp buffers over the window
//   accumulate    num_kq += W_k y_kq into per-lane FP32 registers, combined per CTA in FP64
//
// Each pair streams its images through a ring of ns slots filled by bulk copies; a slot is
// refilled after the first pair barrier, by which both warps hold their rows in registers.
#pragma once
#include "common.cuh"

namespace mra {

constexpr int kV6Threads = 512;  // 8 warp pairs

__device__ __forceinline__ int v6_mod(int a, int L, float invL) {
  int m = a - __float2int_rz((float)a * invL) * L;
  if (m < 0) m += L;
  if (m >= L) m -= L;
  return m;
}
__device__ __forceinline__ int v6_f2ord(float v) {
  const int i = __float_as_int(v);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float v6_ord2f(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }
// Barrier of the 64 threads of one warp pair (named barrier id 1 + pair).
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }
// The same barrier, returning whether p holds in every thread of the pair.
__device__ __forceinline__ bool pair_all(int id, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred a, b;\n\t"
      "setp.ne.u32 a, %1, 0;\n\t"
      "bar.red.and.pred b, %2, 64, a;\n\t"
      "selp.u32 %0, 1, 0, b;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id)
      : "memory");
  return r != 0;
}

template <int QV, int MR>
__global__ void __launch_bounds__(kV6Threads, 1) k_sweep_v6(const SweepV6Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = kV6Threads, NW = NT / 32, NP = NW / 2;
  constexpr int row4 = QV * 4;   // float4 per row
  constexpr int RW = 8 * MR;     // rows per warp
  constexpr int TP = RW / 2;     // row pairs per warp
  constexpr unsigned FULL = 0xffffffffu;
  if (a.ctrl->done) return;
  const bool want_ysq = (a.ctrl->iter == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pr = warp >> 1, h = warp & 1;  // pair, half
  const int r = lane >> 2, j = lane & 3;
  const int K = a.K, L = a.L, Lw = a.Lw, NU = a.NU, M = a.M, ns = a.ns;
  const float invL = 1.0f / (float)L;
  const int bid = 1 + pr;

  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.off_bar) + pr * ns;
  unsigned char* ring = smem + a.off_ring + (size_t)pr * ns * a.slot_bytes;
  const float4* tab4 = reinterpret_cast<const float4*>(smem + a.off_tab);  // [16 MR / 2][32] row pairs
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);    // [L]
  const float* lrs = reinterpret_cast<const float*>(smem + a.off_lr);      // [Lw]
  const int2* uab = reinterpret_cast<const int2*>(smem + a.off_units);     // [32]
  float2* cbw = reinterpret_cast<float2*>(smem + a.off_cb) + warp * RW;    // this warp's c_k
  float2* xp = reinterpret_cast<float2*>(smem + a.off_xp) + pr * 64;       // [2][32] pass-1 partials
  float2* xq = reinterpret_cast<float2*>(smem + a.off_xq) + pr * 8;        // [2][4] pass-2 partials
  float* pv = reinterpret_cast<float*>(smem + a.off_pv) + (size_t)pr * 2 * a.sp;  // [2][sp] general path
  float* sb = reinterpret_cast<float*>(smem + a.off_sb) + (size_t)warp * a.sp;    // [sp] general path
  float* wlw = reinterpret_cast<float*>(smem + a.off_wl) + (size_t)pr * a.sp;     // [sp] W_t, warp 0 only

  // ---- shared tables
  {
    float4* tw4 = reinterpret_cast<float4*>(smem + a.off_tab);
    for (int i = tid; i < 8 * MR * 32; i += NT) {  // row pair t holds rows 2t + 1 and 2t + 2
      const int t = i >> 5, u = i & 31;
      const int k0 = 2 * t + 1, k1 = 2 * t + 2;
      float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
      if (u < NU) {
        if (k0 <= K) v0 = a.tu[k0 * a.nup + u];
        if (k1 <= K) v1 = a.tu[k1 * a.nup + u];
      }
      tw4[i] = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    float* lrw = reinterpret_cast<float*>(smem + a.off_lr);
    for (int i = tid; i < Lw; i += NT) lrw[i] = a.logrho32[i];
    int2* uw = reinterpret_cast<int2*>(smem + a.off_units);
    for (int i = tid; i < 32; i += NT) uw[i] = i < NU ? a.units[i] : make_int2(0, -1);
    float* wl0 = reinterpret_cast<float*>(smem + a.off_wl);
    for (int i = tid; i < NP * a.sp; i += NT) wl0[i] = 0.f;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + a.off_bar);
    if (tid < NP * ns) mbar_init(&bars[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();

  // ---- per-lane constants: rows, x, the pass-2 table entries of distance j
  int krow[MR], kld[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    krow[m] = 1 + RW * h + 8 * m + r;
    kld[m] = min(krow[m], K) * row4 + j;
  }
  float4 xr[MR][QV];
  float2 tdr[MR];
  {
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const bool ok = krow[m] <= K;
#pragma unroll
      for (int u = 0; u < QV; ++u) xr[m][u] = ok ? xg[krow[m] * row4 + j + 4 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
      tdr[m] = (ok && j < a.nd) ? a.td[krow[m] * a.nd + j] : make_float2(0.f, 0.f);
    }
  }
  // pass 1: lane owns mirror unit u = lane (window indices ia and ib, ib absent: -inf)
  int ia = 0x3fffffff, ib = 0x3fffffff;
  float lra = -INFINITY, lrb = -INFINITY;
  const bool uact = lane < NU;
  if (uact) {
    const int2 ab = uab[lane];
    ia = ab.x;
    lra = lrs[ab.x];
    if (ab.y >= 0) ib = ab.y, lrb = lrs[ab.y];
  }
  const float4* tcol = tab4 + TP * h * 32 + lane;

  const int gp = blockIdx.x * NP + pr, GP = gridDim.x * NP;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  auto issue = [&](int im, int st) {
    if (im >= a.N) return;
    mbar_arrive_expect_tx(&full[st], img_bytes);
    bulk_g2s(ring + (size_t)st * a.slot_bytes, a.y + (size_t)im * M, img_bytes, &full[st]);
  };
  if (h == 0 && lane == 0)
    for (int s = 0; s < ns; ++s) issue(gp + s * GP, s);
  auto load_shift = [&](int im) -> int {
    if (!a.shift || im >= a.N) return 0;
    int s = a.shift[im];
    if (s < 0 || s >= L) {
      s %= L;
      if (s < 0) s += L;
    }
    return s;
  };

  float4 acc[MR][QV];
#pragma unroll
  for (int m = 0; m < MR; ++m)
#pragma unroll
    for (int u = 0; u < QV; ++u) acc[m][u] = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f);  // row 0 (warp 0, lanes < row4)
  const bool row0 = h == 0 && lane < row4;
  double ll_acc = 0.0, ysq_acc = 0.0;
  const float two_beta = a.two_beta;
  int sj_next = load_shift(gp);

  int st = 0;
  uint32_t parity = 0;
  for (int it = 0; gp + it * GP < a.N; ++it, st = st + 1 == ns ? 0 : st + 1, parity ^= (st == 0)) {
    const int img = gp + it * GP;
    const int sj = sj_next;
    sj_next = load_shift(img + GP);
    const bool ok = mbar_wait_bounded(&full[st], parity);
    const float4* y4 = reinterpret_cast<const float4*>(ring + (size_t)st * a.slot_bytes);

    // ---- this warp's rows of y into registers; row 0 straight into its accumulator
    // rows beyond K read row K: their x is zero (no correlation) and their sums are never stored
    float4 yv[MR][QV];
#pragma unroll
    for (int m = 0; m < MR; ++m)
#pragma unroll
      for (int u = 0; u < QV; ++u) yv[m][u] = y4[kld[m] + 4 * u];
    float sq = 0.f;
    if (row0) {
      const float4 y0 = y4[lane];
      acc0.x += y0.x; acc0.y += y0.y; acc0.z += y0.z; acc0.w += y0.w;
      if (want_ysq) sq = y0.x * y0.x + y0.y * y0.y + y0.z * y0.z + y0.w * y0.w;
    }

    // ---- correlation c_k = sum_q conj(y_kq) x_kq
    float2 c[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      float cr = 0.f, ci = 0.f;
#pragma unroll
      for (int u = 0; u < QV; ++u) {
        const float4 yq = yv[m][u], xq4 = xr[m][u];
        cr = fmaf(yq.x, xq4.x, cr); cr = fmaf(yq.y, xq4.y, cr);
        cr = fmaf(yq.z, xq4.z, cr); cr = fmaf(yq.w, xq4.w, cr);
        ci = fmaf(yq.x, xq4.y, ci); ci = fmaf(-yq.y, xq4.x, ci);
        ci = fmaf(yq.z, xq4.w, ci); ci = fmaf(-yq.w, xq4.z, ci);
        if (want_ysq && krow[m] <= K) {
          sq = fmaf(yq.x, yq.x, sq); sq = fmaf(yq.y, yq.y, sq);
          sq = fmaf(yq.z, yq.z, sq); sq = fmaf(yq.w, yq.w, sq);
        }
      }
      cr += __shfl_xor_sync(FULL, cr, 1);
      ci += __shfl_xor_sync(FULL, ci, 1);
      cr += __shfl_xor_sync(FULL, cr, 2);
      ci += __shfl_xor_sync(FULL, ci, 2);
      c[m] = make_float2(cr, ci);
    }
    if (want_ysq) {
      const float t = warp_sum(sq);
      if (lane == 0) ysq_acc += (double)t;
    }
    // ---- pass 1: this warp's partial over its rows of c_k e^{-i k theta_hat_j} (the alignment)
    if (j == 0) {
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        float2 cv = c[m];
        if (a.shift) cv = cmul(cv, tfs[v6_mod(krow[m] * sj, L, invL)]);
        cbw[8 * m + r] = cv;
      }
    }
    __syncwarp();
    {
      const float4* cb4 = reinterpret_cast<const float4*>(cbw);
      float2 ab0 = make_float2(0.f, 0.f), ab1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < TP; ++t) {
        const float4 cc = cb4[t];  // local rows 2t and 2t + 1
        const float4 tv = tcol[t * 32];  // zero beyond the last unit
        ab0 = __ffma2_rn(make_float2(cc.x, cc.y), make_float2(tv.x, tv.y), ab0);
        ab1 = __ffma2_rn(make_float2(cc.z, cc.w), make_float2(tv.z, tv.w), ab1);
      }
      xp[h * 32 + lane] = __fadd2_rn(ab0, ab1);
    }
    // first pair barrier: both partials written, both warps' rows of y in registers
    if (!pair_all(bid, ok)) {
      if (h == 0 && lane == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        int s2 = st;
        uint32_t p2 = parity;
        for (int s = 0; s < ns; ++s) {  // drain this pair's copies still in flight
          if (img + s * GP < a.N) mbar_wait_bounded(&full[s2], p2);
          if (++s2 == ns) s2 = 0, p2 ^= 1u;
        }
      }
      break;
    }
    if (h == 0 && lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(img + ns * GP, st);
    }
    const float2 AB = __fadd2_rn(xp[lane], xp[32 + lane]);  // the same order in both warps
    const float sa1 = fmaf(two_beta, AB.x - AB.y, lra);  // offset +o (or the unit's only offset)
    const float sb1 = fmaf(two_beta, AB.x + AB.y, lrb);  // offset -o
    int p, D;
    float vref;
    {
      const float v = fmaxf(sa1, sb1);
      const int li = sa1 > sb1 ? ia : sb1 > sa1 ? ib : min(ia, ib);
      const int kmax = __reduce_max_sync(FULL, v6_f2ord(v));
      int pk = __reduce_min_sync(FULL, v6_f2ord(v) == kmax ? li : 0x7fffffff);
      if (pk >= Lw) pk = 0;  // only if every log-weight is -inf
      vref = v6_ord2f(kmax);
      const float thr = vref - 40.f;
      int lo = pk, hi = pk;
      if (sa1 >= thr) lo = min(lo, ia), hi = max(hi, ia);
      if (sb1 >= thr) lo = min(lo, ib), hi = max(hi, ib);
      lo = __reduce_min_sync(FULL, lo);
      hi = __reduce_max_sync(FULL, hi);
      p = pk;
      D = max(pk - lo, hi - pk);
    }

    // ---- pass 2: c'_k = c_k e^{-i k (theta_hat_j + theta_l*)}; S(l* +- d) - S(l*) = A_d -+ B_d with
    // A_d = sum c'.x (cos t - 1), B_d = sum c'.y (-sin t), t = 2 pi k d / L.  The same factors rotate W back.
    int op = a.l0m + p + sj;
    if (op >= L) op -= L;
    if (op >= L) op -= L;
    float2 fk[MR], cq[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      fk[m] = tfs[v6_mod(krow[m] * op, L, invL)];
      cq[m] = cmul(c[m], fk[m]);
    }
    const float lr_ref = lrs[p];
    float2 W[MR];
    if (D < 4) {
      // sharp image: lane j holds the distance d = j, summed over the warp's rows, then over the pair
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
      if (r == 0) xq[h * 4 + j] = make_float2(da, db);
      pair_sync(bid);
      {
        const float2 q0 = xq[j], q1 = xq[4 + j];
        da = q0.x + q1.x;
        db = q0.y + q1.y;
      }
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
      const float inv = __frcp_rn(z);
      const float wa = ea * inv, wb = eb * inv;
      if (h == 0) {
        if (r == 0) {
          if (va) wlw[la] += wa;
          if (vb) wlw[lb] += wb;
        }
        if (lane == 0) ll_acc += (double)(vref + (mx + __logf(z)));
        if (a.w_out) {  // every lane of the warp runs the same trip count (the shuffles need all)
          float* wo = a.w_out + (size_t)img * Lw;
          for (int l0 = 0; l0 < Lw; l0 += 32) {
            const int l = l0 + lane, d = l - p;
            const float fa = __shfl_sync(FULL, wa, min(max(d, 0), 3));
            const float fb = __shfl_sync(FULL, wb, min(max(-d, 0), 3));
            if (l < Lw) wo[l] = (d >= 0 && d <= 3) ? fa : (d < 0 && d >= -3) ? fb : 0.f;
          }
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
      // ---- general path: this warp's partial differences within D of the peak, combined over the pair
      // in shared memory; both warps then normalise the same values
      const int nd1 = a.nd - 1;
      for (int d0 = 0; d0 <= D; d0 += 8) {
        constexpr int kT = 2;  // distance slots per lane per chunk
        const int nt = min(kT, (D - d0) / 4 + 1);
        float Ad[kT], Bd[kT];
#pragma unroll
        for (int t = 0; t < kT; ++t) Ad[t] = 0.f, Bd[t] = 0.f;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          if (krow[m] <= K) {
            const float2* tr = a.td + (size_t)krow[m] * a.nd;
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
            float da = Ad[t] - Bd[t], db = Ad[t] + Bd[t];
            da += __shfl_xor_sync(FULL, da, 4);
            db += __shfl_xor_sync(FULL, db, 4);
            da += __shfl_xor_sync(FULL, da, 8);
            db += __shfl_xor_sync(FULL, db, 8);
            da += __shfl_xor_sync(FULL, da, 16);
            db += __shfl_xor_sync(FULL, db, 16);
            const int d = d0 + j + 4 * t;
            if (r == 0 && d <= D) {
              const int la = p + d, lb = p - d;
              if (la < Lw) pv[h * a.sp + la] = da;
              if (d > 0 && lb >= 0) pv[h * a.sp + lb] = db;
            }
          }
        }
      }
      pair_sync(bid);
      auto near = [&](int l) { return l >= p - D && l <= p + D; };
      float mx = -INFINITY;
      for (int l = lane; l < Lw; l += 32) {
        if (near(l)) {
          const float s = fmaf(two_beta, pv[l] + pv[a.sp + l], lrs[l] - lr_ref);
          sb[l] = s;
          mx = fmaxf(mx, s);
        }
      }
      mx = warp_max(mx);
      float z = 0.f;
      for (int l = lane; l < Lw; l += 32) {
        const float e = near(l) ? __expf(sb[l] - mx) : 0.f;
        sb[l] = e;
        z += e;
      }
      z = warp_sum(z);
      const float inv = 1.f / z;
      float* wo = (a.w_out && h == 0) ? a.w_out + (size_t)img * Lw : nullptr;
      for (int l = lane; l < Lw; l += 32) {
        const float w = sb[l] * inv;
        sb[l] = w;
        if (h == 0) wlw[l] += w;
        if (wo) wo[l] = w;
      }
      if (h == 0 && lane == 0) ll_acc += (double)(vref + (mx + __logf(z)));
      __syncwarp();
      // back transform around the peak on the distance units d <= D, this warp's rows
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
      for (int d0 = 0; d0 <= D; d0 += 8) {
        constexpr int kT = 2;
        const int nt = min(kT, (D - d0) / 4 + 1);
#pragma unroll
        for (int t = 0; t < kT; ++t) {
          if (t < nt) {
            const int d = d0 + j + 4 * t;
            const float2 sw = wpair(d);
#pragma unroll
            for (int m = 0; m < MR; ++m) {
              if (krow[m] <= K) {
                const float2 tv = a.td[(size_t)krow[m] * a.nd + min(d, nd1)];
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

    // ---- accumulate W_k y_kq from registers
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const float2 w = W[m];
#pragma unroll
      for (int u = 0; u < QV; ++u) {
        const float4 yq = yv[m][u];
        float4& q = acc[m][u];
        q.x = fmaf(w.x, yq.x, q.x); q.x = fmaf(-w.y, yq.y, q.x);
        q.y = fmaf(w.x, yq.y, q.y); q.y = fmaf(w.y, yq.x, q.y);
        q.z = fmaf(w.x, yq.z, q.z); q.z = fmaf(-w.y, yq.w, q.z);
        q.w = fmaf(w.x, yq.w, q.w); q.w = fmaf(w.y, yq.z, q.w);
      }
    }
  }

  // ---- CTA combination: per-pair FP32 sums through the (now idle) ring, then FP64 partials
  __syncthreads();
  float4* red4 = reinterpret_cast<float4*>(smem + a.off_ring);  // [NP][M/2]
  const int half = M / 2;
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    if (krow[m] <= K) {
#pragma unroll
      for (int u = 0; u < QV; ++u) red4[(size_t)pr * half + krow[m] * row4 + j + 4 * u] = acc[m][u];
    }
  }
  if (row0) red4[(size_t)pr * half + lane] = acc0;
  __syncthreads();
  const int G = a.G, cta = blockIdx.x;
  const float* redf = reinterpret_cast<const float*>(smem + a.off_ring);
  __shared__ double llk0[NW];  // the k = 0 likelihood term, per warp of the first row's columns
  double k0 = 0.0;
  for (int col = tid; col < 2 * M; col += NT) {
    float sum = 0.f;
    for (int w = 0; w < NP; ++w) sum += redf[(size_t)w * 2 * M + col];
    a.part[(size_t)col * G + cta] = (double)sum;
    if (col < 2 * row4 * 2) k0 += (double)sum * (double)reinterpret_cast<const float*>(a.x32)[col];
  }
  k0 = warp_sum_d(k0);
  if (lane == 0) llk0[warp] = k0;
  const float* wl0 = reinterpret_cast<const float*>(smem + a.off_wl);
  for (int l = tid; l < Lw; l += NT) {
    float sum = 0.f;
    for (int w = 0; w < NP; ++w) sum += wl0[w * a.sp + l];
    a.part[(size_t)(2 * M + l) * G + cta] = (double)sum;
  }
  __shared__ double red[2][NW];
  if (lane == 0) red[0][warp] = ll_acc, red[1][warp] = ysq_acc;
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0, tk = 0.0;
    for (int w = 0; w < NW; ++w) t0 += red[0][w], t1 += red[1][w], tk += llk0[w];
    a.part[(size_t)(2 * M + Lw) * G + cta] = t0 + (double)two_beta * tk;
    a.part[(size_t)(2 * M + Lw + 1) * G + cta] = t1;
  }
}

}  // namespace mra

// Instantiation table for one row width QV: MR rows per quad and warp (K <= 16 MR), with at most
// six float4 of y per lane.
#define MRA_SWEEP_V6_CASE(QV, MR) \
  case MR: return SweepV6Launch{k_sweep_v6<QV, MR>, kV6Threads};
#define MRA_SWEEP_V6_TABLE(QV, ...)     \
  namespace mra {                       \
  SweepV6Launch sweep_v6_q##QV(int MR) { \
    switch (MR) {                       \
      __VA_ARGS__                       \
      default: return {nullptr, 0};     \
    }                                   \
  }                                     \
  }
