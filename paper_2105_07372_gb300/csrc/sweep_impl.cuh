// Warp-per-image EM sweep (rows of Q a multiple of 8 coefficients).
//
// Each warp owns a private two-slot shared-memory ring filled by bulk copies
// (one image per copy) and runs an image through every stage with warp-level
// synchronisation only:
//
//   lanes form 8 quads; quad r owns the rows k = r, r+8, r+16, ...; lane j of a
//   quad owns the float4 columns j, j+4, ... of those rows (QV of them per row).
//
//   correlation   c_k = sum_q conj(y_kq) x_kq        quad-local, two xor shuffles
//   forward       S_l = Re sum_k c_k e^{-i k theta_l}, window offsets grouped in
//                 mirror units {+o, -o}: A = sum c.x cos, B = sum c.y sin give
//                 S_{+o} = A - B and S_{-o} = A + B (halves the work)
//   normalise     w_l = exp(s_l - max) / Z over the per-warp s buffer
//   back          W_k = sum_l w_l e^{+i k theta_l} = sum_units (w_+ + w_-) cos + i (w_- - w_+) sin
//   accumulate    num_kq += W_k y_kq into per-lane FP32 registers
//
// The CTA combines its warps' sums once at the end and writes FP64 partials.
#pragma once
#include "common.cuh"

namespace mra {

template <int QV, int MR>
struct SweepV2Shape {
  static constexpr int kThreads = (MR * QV * 4 > 64) ? 256 : 512;
  static constexpr int kWarps = kThreads / 32;
};

constexpr int kUC = 5;  // mirror units per lane per chunk

template <int QV, int MR>
__global__ void __launch_bounds__(SweepV2Shape<QV, MR>::kThreads, 1) k_sweep_v2(const SweepV2Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NT = SweepV2Shape<QV, MR>::kThreads;
  if (a.ctrl->done) return;
  const bool want_ysq = (a.ctrl->iter == 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = a.nwarps;  // <= NT/32 (warps beyond it only join the final reduction)
  const int r = lane >> 2, j = lane & 3;
  const int Kp1 = a.Kp1, L = a.L, Lw = a.Lw, NU = a.NU, NUP = a.NUP, M = a.M;
  const int row4 = QV * 4;  // float4 per row

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);  // [nwarps][2]
  unsigned char* ring = smem + a.off_ring;            // [nwarps][2][slot]
  const float4* xs4 = reinterpret_cast<const float4*>(smem + a.off_x);
  const float2* tus = reinterpret_cast<const float2*>(smem + a.off_tu);  // [Kp1][NUP]
  const float2* tfs = reinterpret_cast<const float2*>(smem + a.off_tf);  // [L]
  const float* lrs = reinterpret_cast<const float*>(smem + a.off_lr);    // [Lw]
  const int2* uab = reinterpret_cast<const int2*>(smem + a.off_units);   // [NUP] (a, b) window indices, b < 0: single
  const int2* lmap = reinterpret_cast<const int2*>(smem + a.off_lmap);   // [Lw] (unit, -1 first offset / +1 mirror)
  float* sbuf = reinterpret_cast<float*>(smem + a.off_s) + warp * a.sp;   // per-warp [Lw]
  float* wlw = reinterpret_cast<float*>(smem + a.off_wl) + warp * a.sp;   // per-warp [Lw]

  // ---- shared tables
  {
    float4* x4w = reinterpret_cast<float4*>(smem + a.off_x);
    const float4* xg = reinterpret_cast<const float4*>(a.x32);
    for (int i = tid; i < M / 2; i += NT) x4w[i] = xg[i];
    float2* tuw = reinterpret_cast<float2*>(smem + a.off_tu);
    for (int i = tid; i < Kp1 * NUP; i += NT) tuw[i] = a.tu[i];
    float2* tfw = reinterpret_cast<float2*>(smem + a.off_tf);
    for (int i = tid; i < L; i += NT) tfw[i] = a.tf32[i];
    float* lrw = reinterpret_cast<float*>(smem + a.off_lr);
    for (int i = tid; i < Lw; i += NT) lrw[i] = a.logrho32[i];
    int2* uw = reinterpret_cast<int2*>(smem + a.off_units);
    int2* lw = reinterpret_cast<int2*>(smem + a.off_lmap);
    for (int i = tid; i < NUP; i += NT) {
      const int2 ab = a.units[i];
      uw[i] = ab;
      if (i < NU && ab.x >= 0 && ab.x < Lw) {
        lw[ab.x] = make_int2(i, -1);
        if (ab.y >= 0 && ab.y < Lw) lw[ab.y] = make_int2(i, 1);
      }
    }
    float* wl0 = reinterpret_cast<float*>(smem + a.off_wl);
    for (int i = tid; i < a.sp * (NT / 32); i += NT) wl0[i] = 0.f;
    if (tid < 2 * nwarps) mbar_init(&bar[tid], 1);
    if (tid == 0) fence_barrier_init();
  }
  __syncthreads();

  const int gw = blockIdx.x * nwarps + warp, GW = gridDim.x * nwarps;
  const uint32_t img_bytes = (uint32_t)M * 8u;
  unsigned char* const slot0 = ring + (size_t)(warp * 2) * a.slot_bytes;  // slot s at slot0 + s * slot_bytes
  uint64_t* mybar = bar + 2 * warp;

  float4 acc[MR][QV];
#pragma unroll
  for (int m = 0; m < MR; ++m)
#pragma unroll
    for (int u = 0; u < QV; ++u) acc[m][u] = make_float4(0.f, 0.f, 0.f, 0.f);
  double ll_acc = 0.0, ysq_acc = 0.0;
  const float two_beta = a.two_beta;

  if (warp < nwarps && lane == 0) {
    if (gw < a.N) {
      mbar_arrive_expect_tx(&mybar[0], img_bytes);
      bulk_g2s(slot0, a.y + (size_t)gw * M, img_bytes, &mybar[0]);
    }
    if (gw + GW < a.N) {
      mbar_arrive_expect_tx(&mybar[1], img_bytes);
      bulk_g2s(slot0 + a.slot_bytes, a.y + (size_t)(gw + GW) * M, img_bytes, &mybar[1]);
    }
  }

  int n = 0;
  for (int img = gw; warp < nwarps && img < a.N; img += GW, ++n) {
    const int s = n & 1;
    const uint32_t parity = (uint32_t)((n >> 1) & 1);
    const bool ok = mbar_wait_bounded(&mybar[s], parity);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        mbar_wait_bounded(&mybar[s], parity);
        if (img + GW < a.N) mbar_wait_bounded(&mybar[s ^ 1], (uint32_t)(((n + 1) >> 1) & 1));
      }
      break;
    }
    unsigned char* const cur = slot0 + s * a.slot_bytes;
    const float4* y4 = reinterpret_cast<const float4*>(cur);

    int sj = 0;
    if (a.shift) {
      sj = a.shift[img] % L;
      if (sj < 0) sj += L;
    }
    const int ph0 = (r * sj) % L, phstep = (8 * sj) % L;

    float2 W[MR];
    if (a.align_only) {
      // weights are exactly 1 at offset 0: W_k = e^{+i k theta_hat_j}
      int ph = ph0;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const float2 t = tfs[ph];
        W[m] = make_float2(t.x, -t.y);
        ph += phstep;
        if (ph >= L) ph -= L;
      }
    } else {
      // ---- correlation
      float2 c[MR];
      float sq = 0.f;
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        const int k = r + 8 * m;
        float cr = 0.f, ci = 0.f;
        if (k < Kp1) {
#pragma unroll
          for (int u = 0; u < QV; ++u) {
            const int p = k * row4 + j + 4 * u;
            const float4 yv = y4[p], xv = xs4[p];
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
        c[m] = make_float2(cr, ci);
      }
      if (want_ysq) {
        sq = warp_sum(sq);
        if (lane == 0) ysq_acc += (double)sq;
      }
      if (a.shift) {  // c_k e^{-i k theta_hat_j}
        int ph = ph0;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          c[m] = cmul(c[m], tfs[ph]);
          ph += phstep;
          if (ph >= L) ph -= L;
        }
      }

      // ---- forward transform over mirror units (chunks of 4 * kUC units).
      // Pass 1 gives FP32 log-weights good enough to find each image's peak rotation l*.
      // Pass 2 re-expresses every quad partial relative to the quad partial of l* before
      // the cross-quad sums, so that near the peak (where the weights are not negligible)
      // the sums add small numbers: s is stored relative to s(l*).
      auto partials = [&](int u0, float (&A)[kUC], float (&Bv)[kUC]) {
#pragma unroll
        for (int t = 0; t < kUC; ++t) A[t] = 0.f, Bv[t] = 0.f;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          const int k = r + 8 * m;
          if (k < Kp1) {
            const float2 cc = c[m];
            const float2* trow = tus + k * NUP + u0 + j;
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              const float2 tv = trow[4 * t];
              A[t] = fmaf(cc.x, tv.x, A[t]);
              Bv[t] = fmaf(cc.y, tv.y, Bv[t]);
            }
          }
        }
      };
      auto quad_sum = [&](float v) {
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        return v;
      };
      auto store_rel = [&](int u0, const float (&Da)[kUC], const float (&Db)[kUC], float lr_ref) {
        if (r == 0) {
#pragma unroll
          for (int t = 0; t < kUC; ++t) {
            const int u = u0 + j + 4 * t;
            if (u < NU) {
              const int2 ab = uab[u];
              sbuf[ab.x] = fmaf(two_beta, Da[t], lrs[ab.x] - lr_ref);
              if (ab.y >= 0) sbuf[ab.y] = fmaf(two_beta, Db[t], lrs[ab.y] - lr_ref);
            }
          }
        }
      };
      float vref;  // FP32 log-weight at l* (absolute)
      if (NUP == 4 * kUC) {
        float A[kUC], Bv[kUC];
        partials(0, A, Bv);
        float bv = -INFINITY;
        int bl = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < kUC; ++t) {
          const int u = j + 4 * t;
          const float At = quad_sum(A[t]), Bt = quad_sum(Bv[t]);
          if (u < NU) {
            const int2 ab = uab[u];
            const float sa = fmaf(two_beta, At - Bt, lrs[ab.x]);
            if (sa > bv || (sa == bv && ab.x < bl)) bv = sa, bl = ab.x;
            if (ab.y >= 0) {
              const float sb = fmaf(two_beta, At + Bt, lrs[ab.y]);
              if (sb > bv || (sb == bv && ab.y < bl)) bv = sb, bl = ab.y;
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
        vref = bv;
        const int2 um = lmap[bl];  // (unit, -1 for its first offset / +1 for the mirror)
        const int tstar = um.x >> 2, jstar = um.x & 3;
        float pa = A[0], pb = Bv[0];
#pragma unroll
        for (int t = 1; t < kUC; ++t)
          if (t == tstar) pa = A[t], pb = Bv[t];
        float pr = um.y < 0 ? pa - pb : pa + pb;
        pr = __shfl_sync(0xffffffffu, pr, (lane & ~3) | jstar);
        float Da[kUC], Db[kUC];
#pragma unroll
        for (int t = 0; t < kUC; ++t) {
          Da[t] = quad_sum((A[t] - Bv[t]) - pr);
          Db[t] = quad_sum((A[t] + Bv[t]) - pr);
        }
        store_rel(0, Da, Db, lrs[bl]);
      } else {
        for (int u0 = 0; u0 < NUP; u0 += 4 * kUC) {  // pass 1 into the per-warp buffer
          float A[kUC], Bv[kUC];
          partials(u0, A, Bv);
          float At[kUC], Bt[kUC];
#pragma unroll
          for (int t = 0; t < kUC; ++t) At[t] = quad_sum(A[t]), Bt[t] = quad_sum(Bv[t]);
          if (r == 0) {
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              const int u = u0 + j + 4 * t;
              if (u < NU) {
                const int2 ab = uab[u];
                sbuf[ab.x] = fmaf(two_beta, At[t] - Bt[t], lrs[ab.x]);
                if (ab.y >= 0) sbuf[ab.y] = fmaf(two_beta, At[t] + Bt[t], lrs[ab.y]);
              }
            }
          }
        }
        __syncwarp();
        float bv = -INFINITY;
        int bl = 0x7fffffff;
        for (int l = lane; l < Lw; l += 32) {
          const float v = sbuf[l];
          if (v > bv) bv = v, bl = l;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
          if (ov > bv || (ov == bv && ol < bl)) bv = ov, bl = ol;
        }
        if (bl >= Lw) bl = 0;
        vref = bv;
        const int2 um = lmap[bl];
        float pa = 0.f, pb = 0.f;  // the reference's quad partial, same arithmetic as partials()
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          const int k = r + 8 * m;
          if (k < Kp1) {
            const float2 tv = tus[k * NUP + um.x];
            pa = fmaf(c[m].x, tv.x, pa);
            pb = fmaf(c[m].y, tv.y, pb);
          }
        }
        const float pr = um.y < 0 ? pa - pb : pa + pb;
        const float lr_ref = lrs[bl];
        for (int u0 = 0; u0 < NUP; u0 += 4 * kUC) {  // pass 2 where the weights matter
          bool sig = false;
#pragma unroll
          for (int t = 0; t < kUC; ++t) {
            const int u = u0 + j + 4 * t;
            if (u < NU) {
              const int2 ab = uab[u];
              sig |= sbuf[ab.x] >= vref - 40.f;
              if (ab.y >= 0) sig |= sbuf[ab.y] >= vref - 40.f;
            }
          }
          sig = __any_sync(0xffffffffu, sig);
          __syncwarp();
          if (sig) {
            float A[kUC], Bv[kUC], Da[kUC], Db[kUC];
            partials(u0, A, Bv);
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              Da[t] = quad_sum((A[t] - Bv[t]) - pr);
              Db[t] = quad_sum((A[t] + Bv[t]) - pr);
            }
            store_rel(u0, Da, Db, lr_ref);
          } else if (r == 0) {
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              const int u = u0 + j + 4 * t;
              if (u < NU) {
                const int2 ab = uab[u];
                sbuf[ab.x] -= vref;
                if (ab.y >= 0) sbuf[ab.y] -= vref;
              }
            }
          }
        }
      }
      __syncwarp();

      // ---- normalisation over the window
      float mx = -INFINITY;
      for (int l = lane; l < Lw; l += 32) mx = fmaxf(mx, sbuf[l]);
      mx = warp_max(mx);
      float z = 0.f;
      for (int l = lane; l < Lw; l += 32) {
        const float e = expf(sbuf[l] - mx);
        sbuf[l] = e;
        z += e;
      }
      z = warp_sum(z);
      const float inv = 1.f / z;
      float* wo = a.w_out ? a.w_out + (size_t)img * Lw : nullptr;
      for (int l = lane; l < Lw; l += 32) {
        const float w = sbuf[l] * inv;
        sbuf[l] = w;
        wlw[l] += w;
        if (wo) wo[l] = w;
      }
      if (lane == 0) ll_acc += (double)vref + (double)mx + (double)logf(z);
      __syncwarp();

      // ---- back transform
#pragma unroll
      for (int m = 0; m < MR; ++m) W[m] = make_float2(0.f, 0.f);
      for (int u0 = 0; u0 < NUP; u0 += 4 * kUC) {
        float sw[kUC], dw[kUC];
#pragma unroll
        for (int t = 0; t < kUC; ++t) {
          const int u = u0 + j + 4 * t;
          float wa = 0.f, wb = 0.f;
          if (u < NU) {
            const int2 ab = uab[u];
            wa = sbuf[ab.x];
            wb = ab.y >= 0 ? sbuf[ab.y] : 0.f;
          }
          sw[t] = wa + wb;
          dw[t] = wb - wa;
        }
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          const int k = r + 8 * m;
          if (k < Kp1) {
            const float2* trow = tus + k * NUP + u0 + j;
#pragma unroll
            for (int t = 0; t < kUC; ++t) {
              const float2 tv = trow[4 * t];
              W[m].x = fmaf(sw[t], tv.x, W[m].x);
              W[m].y = fmaf(dw[t], tv.y, W[m].y);
            }
          }
        }
      }
#pragma unroll
      for (int m = 0; m < MR; ++m) {
        W[m].x += __shfl_xor_sync(0xffffffffu, W[m].x, 1);
        W[m].y += __shfl_xor_sync(0xffffffffu, W[m].y, 1);
        W[m].x += __shfl_xor_sync(0xffffffffu, W[m].x, 2);
        W[m].y += __shfl_xor_sync(0xffffffffu, W[m].y, 2);
      }
      if (a.shift) {  // W_k e^{+i k theta_hat_j}
        int ph = ph0;
#pragma unroll
        for (int m = 0; m < MR; ++m) {
          W[m] = cmul_conj_b(W[m], tfs[ph]);
          ph += phstep;
          if (ph >= L) ph -= L;
        }
      }
    }

    // ---- accumulate W_k y_kq
#pragma unroll
    for (int m = 0; m < MR; ++m) {
      const int k = r + 8 * m;
      if (k < Kp1) {
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
    // slot s may be refilled once every lane has finished reading it
    __syncwarp();
    if (lane == 0 && img + 2 * GW < a.N) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(&mybar[s], img_bytes);
      bulk_g2s(cur, a.y + (size_t)(img + 2 * GW) * M, img_bytes, &mybar[s]);
    }
  }

  // ---- CTA combination: per-warp FP32 sums through the (now idle) ring, then FP64 partials
  __syncthreads();
  float4* red4 = reinterpret_cast<float4*>(ring);  // [NT/32][M/2]
  const int half = M / 2;
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int k = r + 8 * m;
    if (k < Kp1) {
#pragma unroll
      for (int u = 0; u < QV; ++u) red4[(size_t)warp * half + k * row4 + j + 4 * u] = acc[m][u];
    }
  }
  __syncthreads();
  const int G = a.G, cta = blockIdx.x;
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

}  // namespace mra

// Instantiation table for one row width QV: MR = 1..7 rows per quad.
#define MRA_SWEEP_V2_TABLE(QV)                                                                   \
  namespace mra {                                                                               \
  SweepV2Launch sweep_v2_q##QV(int MR) {                                                        \
    switch (MR) {                                                                                \
      case 1: return {k_sweep_v2<QV, 1>, SweepV2Shape<QV, 1>::kThreads};                         \
      case 2: return {k_sweep_v2<QV, 2>, SweepV2Shape<QV, 2>::kThreads};                         \
      case 3: return {k_sweep_v2<QV, 3>, SweepV2Shape<QV, 3>::kThreads};                         \
      case 4: return {k_sweep_v2<QV, 4>, SweepV2Shape<QV, 4>::kThreads};                         \
      case 5: return {k_sweep_v2<QV, 5>, SweepV2Shape<QV, 5>::kThreads};                         \
      case 6: return {k_sweep_v2<QV, 6>, SweepV2Shape<QV, 6>::kThreads};                         \
      case 7: return {k_sweep_v2<QV, 7>, SweepV2Shape<QV, 7>::kThreads};                         \
      default: return {nullptr, 0};                                                              \
    }                                                                                            \
  }                                                                                              \
  }
