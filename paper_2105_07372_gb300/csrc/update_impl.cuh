// The EM finalize of one iteration (Eq. coefficients_update, the rho update of Algorithm Synch-EM with
// its gamma-weighted prior, App. C, and the stopping rule): state a_{t+1}, rho_{t+1}, the
// log-likelihood at a_t and the step, from the FP64 column totals of the sweep.
#pragma once
#include "common.cuh"

namespace mra {

struct UpdateArgs {
  int N, Kp1, Q, M, L, Lw;
  double sigma2, beta, gamma, tol;
  double ll_const;  // N M log(pi sigma2), computed on the host (an FP64 log is slow on the device)
  int update_rho, max_iters;
  const double* tot;  // [cols + 8]; tot[cols] keeps sum_j ||y_j||^2 from the first iteration
  int cols;
  double2* x64;
  float2* x32;
  const double* inv_den;
  double* rho64;
  float* logrho32;
  const double* rhobar64;
  const double2* tf64;
  const float2* tf32;
  Ctrl* ctrl;
  double* stats;    // [T][2] or null
  double2* x_traj;  // [T][M] or null
  double2* x_out;
  double* log_rho_out;
  double* loglik_out;
  double* step_out;
};

// Block-wide FP64 sum, fixed order; red needs 33 slots.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum_d(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Shared memory of the update: xn [M] double2, t64 [L] double2, t32 [L] float2, d32 [Kp1] float2,
// sc [L] float, then xf [M] float4 (a_{t+1}, a_t in FP32) at a 16-byte boundary.
__host__ __device__ inline int update_xf_offset(int M, int L, int Kp1) {
  return (16 * M + 28 * L + 8 * Kp1 + 15) & ~15;
}

__device__ __forceinline__ float block_sum_f(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    float t = lane < nw ? red[lane] : 0.f;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// One CTA: a_{t+1}, rho_{t+1}, log-likelihood at a_t, step; state update.  FP64 arithmetic is
// slow on this part (one FP64 warp instruction holds the SM's FP64 pipe for many cycles), so
// FP64 is kept to the state a_{t+1} = num / (N + sigma^2 Gamma^-1) and the final likelihood
// sum; norms, rho and the step run in FP32 (the step as a direct sum of squares, which has no
// cancellation, to relative accuracy ~1e-6).
constexpr int kUpdateThreads = 512;

// A device function, so that the batched persistent kernel runs the same update for each instance;
// k_finalize runs it in the last of its CTAs (kUpdateThreads threads).
__device__ __forceinline__ void update_body(const UpdateArgs& a) {
  extern __shared__ __align__(16) unsigned char usmem[];
  // the state, the totals and the control words may come from other CTAs of a persistent launch:
  // read them through L2
  if (__ldcg(&a.ctrl->done)) return;
  double2* xn = reinterpret_cast<double2*>(usmem);            // [M]
  double2* t64 = xn + a.M;                                      // [L]  (unused: kept for layout)
  float2* t32 = reinterpret_cast<float2*>(t64 + a.L);          // [L]
  float2* d32 = t32 + a.L;                                      // [Kp1]
  float* sc = reinterpret_cast<float*>(d32 + a.Kp1);           // [L]
  float4* xf = reinterpret_cast<float4*>(usmem + update_xf_offset(a.M, a.L, a.Kp1));  // [M]
  __shared__ float fred[33];
  __shared__ double ysq_total;
  __shared__ int ncand;
  __shared__ int cand[16];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int iter = __ldcg(&a.ctrl->iter);
  if (tid == 0) ncand = 0;
  for (int l = tid; l < a.L; l += nt) t32[l] = a.tf32[l];

  float nx_old = 0.f;
  for (int e = tid; e < a.M; e += nt) {
    const double2 xo = __ldcg(a.x64 + e);
    const double id = a.inv_den[e];
    const double2 v = make_double2(__ldcg(a.tot + 2 * e) * id, __ldcg(a.tot + 2 * e + 1) * id);
    xn[e] = v;
    xf[e] = make_float4((float)v.x, (float)v.y, (float)xo.x, (float)xo.y);
    nx_old = fmaf((float)xo.x, (float)xo.x, fmaf((float)xo.y, (float)xo.y, nx_old));
  }
  nx_old = block_sum_f(nx_old, fred);
  if (tid == 0) {
    double* keep = const_cast<double*>(a.tot) + a.cols;
    const double kv = iter == 0 ? __ldcg(a.tot + 2 * a.M + a.Lw + 1) : __ldcg(keep);
    if (iter == 0) keep[0] = kv;
    ysq_total = kv;
  }
  // d_k = sum_q conj(a_{t+1,kq}) a_{t,kq} (FP32, ranks the rotations), one warp per row
  for (int k = warp; k < a.Kp1; k += nw) {
    float dr = 0.f, di = 0.f;
    for (int q = lane; q < a.Q; q += 32) {
      const float4 v = xf[k * a.Q + q];
      dr = fmaf(v.x, v.z, fmaf(v.y, v.w, dr));
      di = fmaf(v.x, v.w, fmaf(-v.y, v.z, di));
    }
    dr = warp_sum(dr);
    di = warp_sum(di);
    if (lane == 0) d32[k] = make_float2(dr, di);
  }
  __syncthreads();

  // rho update (one warp: the window is short)
  if (warp == 0) {
    if (a.update_rho) {
      float v = 0.f;
      for (int l = lane; l < a.Lw; l += 32) v += (float)(__ldcg(a.tot + 2 * a.M + l) + a.gamma * a.rhobar64[l]);
      const float inv = 1.f / warp_sum(v);
      for (int l = lane; l < a.Lw; l += 32) {
        const float r = (float)(__ldcg(a.tot + 2 * a.M + l) + a.gamma * a.rhobar64[l]) * inv;
        a.rho64[l] = (double)r;
        a.logrho32[l] = logf(r);  // -inf for an empty bin
        if (a.log_rho_out) a.log_rho_out[l] = (double)logf(r);
      }
    } else if (a.log_rho_out) {
      for (int l = lane; l < a.Lw; l += 32) a.log_rho_out[l] = (double)logf((float)__ldcg(a.rho64 + l));
    }
  }

  // step: rank the L rotations in FP32
  float dmag = 0.f;
  for (int k = 0; k < a.Kp1; ++k) dmag += fabsf(d32[k].x) + fabsf(d32[k].y);
  float best = -INFINITY;
  for (int l = tid; l < a.L; l += nt) {
    float sv = 0.f;
    int m = 0;
    for (int k = 0; k < a.Kp1; ++k) {
      const float2 t = t32[m], dv = d32[k];
      sv = fmaf(dv.x, t.x, fmaf(-dv.y, t.y, sv));
      m += l;
      if (m >= a.L) m -= a.L;
    }
    sc[l] = sv;
    best = fmaxf(best, sv);
  }
  best = warp_max(best);
  if (lane == 0) fred[warp] = best;
  __syncthreads();
  float gbest = -INFINITY;
  for (int w = 0; w < nw; ++w) gbest = fmaxf(gbest, fred[w]);
  const float thr = gbest - (1e-5f * dmag + 1e-30f);
  for (int l = tid; l < a.L; l += nt) {
    if (sc[l] >= thr) {
      const int slot = atomicAdd(&ncand, 1);
      if (slot < 16) cand[slot] = l;
    }
  }
  __syncthreads();
  const int nc = min(ncand, 16);
  // ||a_{t+1} - e^{-2 pi i k l / L} a_t||^2 of the candidates, summed directly in FP32
  float step = INFINITY;
  for (int ci = 0; ci < nc; ++ci) {
    const int l = cand[ci];
    float part = 0.f;
    for (int e = tid; e < a.M; e += nt) {
      const int k = e / a.Q;
      const float2 t = t32[(int)(((long long)k * l) % a.L)];
      const float4 v = xf[e];
      const float dr = v.x - (v.z * t.x - v.w * t.y);
      const float di = v.y - (v.z * t.y + v.w * t.x);
      part = fmaf(dr, dr, fmaf(di, di, part));
    }
    step = fminf(step, block_sum_f(part, fred));
  }
  step = fmaxf(step, 0.f);

  // state
  for (int e = tid; e < a.M; e += nt) {
    const double2 v = xn[e];
    a.x64[e] = v;
    a.x32[e] = make_float2((float)v.x, (float)v.y);
    if (a.x_traj) a.x_traj[(size_t)iter * a.M + e] = v;
    if (a.x_out) a.x_out[e] = v;
  }
  if (tid == 0) {
    const double ll =
        __ldcg(a.tot + 2 * a.M + a.Lw) - a.beta * ysq_total - (double)a.N * a.beta * (double)nx_old - a.ll_const;
    if (a.stats) {
      a.stats[2 * iter] = ll;
      a.stats[2 * iter + 1] = (double)step;
    }
    if (a.loglik_out) *a.loglik_out = ll;
    if (a.step_out) *a.step_out = (double)step;
    const int nit = iter + 1;
    a.ctrl->iter = nit;
    if ((a.tol > 0.0 && (double)step < a.tol) || nit >= a.max_iters) a.ctrl->done = 1;
  }
}



// tot[col] = sum_g part[col][g] in FP64, one warp per column, fixed summation order.
__device__ __forceinline__ void reduce_cols_warp(const double* part, int G, int col, double* tot) {
  const int lane = threadIdx.x & 31;
  const double* p = part + (size_t)col * G;
  double s = 0.0;
  for (int g = lane; g < G; g += 32) s += __ldcg(p + g);
  s = warp_sum_d(s);
  if (lane == 0) tot[col] = s;
}

}  // namespace mra
