// Windowed, prior-weighted EM for 2-D MRA (Algorithm Synch-EM) on sm_103a.
//
// One EM iteration is one pass over the observations y (the fused sweep), an
// FP64 cross-CTA reduction and a one-CTA update:
//
//   sweep   per image j (tile of B images staged in shared memory by bulk copies):
//             c_jk  = sum_q conj(y_jkq) x_kq                     (E-step distance, cross term)
//             S_jl  = Re sum_k c_jk e^{-i k theta_l}, l in window
//             s_jl  = log rho_l + (2/sigma^2) S_jl                (Eq. weights_2d_em up to a j-constant)
//             w_jl  = exp(s_jl - m_j) / Z_j                       (normalisation over the window)
//             W_jk  = sum_l w_jl e^{+i k theta_l}
//             num_kq += W_jk y_jkq,  W[l] += w_jl,  sum_j (m_j + log Z_j)   (M-step numerator, W_t)
//   reduce  FP64 sum of the per-CTA partials (deterministic order)
//   update  a_{t+1} = num / (N + sigma^2 Gamma^{-1})                   (Eq. coefficients_update)
//           rho_{t+1} = (W + gamma rho_bar) / sum                       (prior-weighted rho update)
//           step = min_l ||a_{t+1} - e^{-2 pi i k l / L} a_t||^2          (stopping rule)
//
// Alignment by estimated shifts is folded in as a per-(image, k) phase on
// c_jk and W_jk; y itself is read once per iteration and never rewritten.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "batched.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace mra {

// ============================================================================ device info
// Kernel dynamic shared-memory limits only grow: the limit belongs to the kernel and is
// shared by every call and every captured graph node that launches it, so lowering it
// for one call could break an earlier node of a graph that is still to run.
int raise_smem_limit(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limit;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRA_ECUDA;
  std::lock_guard<std::mutex> g(mu);
  int& cur = limit[{dev, fn}];
  if (bytes <= cur) return MRA_OK;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return MRA_ECUDA;
  cur = bytes;
  return MRA_OK;
}

int dev_info(DevInfo* out) {
  static DevInfo cache[64];
  static bool have[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MRA_ECUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!have[dev]) {
    int sms = 0, smem = 0, smem_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MRA_ECUDA;
    if (cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return MRA_ECUDA;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
      return MRA_ECUDA;
    cache[dev].sms = sms;
    cache[dev].max_smem_optin = smem;
    cache[dev].smem_per_sm = smem_sm;
    have[dev] = true;
  }
  *out = cache[dev];
  return MRA_OK;
}

int sweep_grid() {
  DevInfo d;
  if (dev_info(&d) != MRA_OK) return -1;
  return d.sms;  // one persistent CTA per SM (the chunked sweep may run two)
}

// ============================================================================ kernels
struct SetupArgs {
  int N, Kp1, Q, M, L, Lw, l0, twp, kp4;
  double sigma2;
  double step;  // spacing of the window's rotations in grid units (1 = the grid)
  int dense;    // step != 1: window angles 2 pi step (l0 + i) / L off the grid
  const double2* x_in;
  const double* log_rho_in;   // may be null (loglik mode)
  const double* log_rho_bar;  // may be null
  const double* gamma_a_inv;  // may be null
  float2* tf32;
  double2* tf64;
  float2* tw;
  double2* tw64;  // the window twiddles in FP64 (tile sweep)
  float2* x32;
  double2* x64;
  double* inv_den;
  float* logrho32;
  double* rho64;
  double* rhobar64;
  int2* units;  // [nup]
  float2* tu;   // [Kp1][nup]
  float2* td;   // [Kp1][nd]
  int nu, nup, nd;
  Ctrl* ctrl;
};

// Twiddles T[m] = e^{-2 pi i m / L} (FP64 and FP32), the state in FP32/FP64, 1/(N + sigma^2 Gamma^-1).
__global__ void k_setup(const SetupArgs a) {
  const int n = max(max(a.L, a.M), a.Lw);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < a.L) {
      double s, c;
      sincospi(2.0 * (double)i / (double)a.L, &s, &c);
      a.tf64[i] = make_double2(c, -s);
      a.tf32[i] = make_float2((float)c, (float)-s);
    }
    if (i < a.M) {
      double2 x = a.x_in[i];
      a.x64[i] = x;
      a.x32[i] = make_float2((float)x.x, (float)x.y);
      double g = a.gamma_a_inv ? a.gamma_a_inv[i] : 0.0;
      a.inv_den[i] = 1.0 / ((double)a.N + a.sigma2 * g);
    }
    if (i < a.Lw) {
      if (a.log_rho_in) {
        // same derivation as the update kernel, so that a run resumed from its exported state
        // continues bit for bit
        const double lr = a.log_rho_in[i];
        const double r = exp(lr);
        a.rho64[i] = r;
        a.logrho32[i] = r > 1e-30 ? logf((float)r) : (float)lr;
      }
      a.rhobar64[i] = a.log_rho_bar ? exp(a.log_rho_bar[i]) : 0.0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->status = MRA_OK;
    a.ctrl->done = 0;
    a.ctrl->iter = 0;
    a.ctrl->sched[0] = 0;
    a.ctrl->sched[1] = 0;
    a.ctrl->fin = 0;
  }
}

// e^{-i k theta} at window position pos of a dense window, theta = 2 pi step pos / L (FP64).
__device__ inline double2 dense_twiddle(int k, int pos, double step, int L) {
  double s, c;
  sincospi(2.0 * step * (double)((long long)k * pos) / (double)L, &s, &c);
  return make_double2(c, -s);
}

// Window twiddles Tw[k][i] = e^{-i k theta_{l0+i}}, zero padded to [kp4][twp], in FP32 and FP64:
// T[(k (l0+i)) mod L] on the grid, the FP64 angle for a dense window.
__global__ void k_setup_tw(const SetupArgs a) {
  const int n = a.kp4 * a.twp;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int k = idx / a.twp, i = idx - k * a.twp;
    double2 v = make_double2(0.0, 0.0);
    if (k < a.Kp1 && i < a.Lw) {
      if (a.dense) {
        v = dense_twiddle(k, a.l0 + i, a.step, a.L);
      } else {
        int off = (a.l0 + i) % a.L;
        if (off < 0) off += a.L;
        v = a.tf64[(int)(((long long)k * off) % a.L)];
      }
    }
    a.tw[idx] = make_float2((float)v.x, (float)v.y);
    a.tw64[idx] = v;
  }
}

// Mirror units of the window (one thread: integer bookkeeping over Lw entries).
// B operand of the split sweep's tensor-core pass 1: row l (window rotation theta_l), columns
// (cos k theta_l, sin k theta_l) for k = 0..K, zero padded to NP rows and KA columns, FP16 in the
// K-major core-matrix layout of tc::op_offset.
__global__ void k_setup_tcb(const SetupArgs a, __half* tcb, int NP, int KA) {
  const int n = NP * KA;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int l = idx / KA, kk = idx - l * KA, k = kk >> 1;
    double v = 0.0;
    if (l < a.Lw && k < a.Kp1) {
      double2 t;  // (cos, -sin) of k theta_l
      if (a.dense) {
        t = dense_twiddle(k, a.l0 + l, a.step, a.L);
      } else {
        int off = (a.l0 + l) % a.L;
        if (off < 0) off += a.L;
        t = a.tf64[(int)(((long long)k * off) % a.L)];
      }
      v = (kk & 1) ? -t.y : t.x;
    }
    *reinterpret_cast<__half*>(reinterpret_cast<unsigned char*>(tcb) + tc::op_offset(l, kk, KA)) =
        __float2half_rn((float)v);
  }
}

__global__ void k_setup_units(const SetupArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int nu = window_units(a.L, a.Lw, a.l0, a.dense != 0, a.units);
    for (int u = nu; u < a.nup; ++u) a.units[u] = make_int2(0, -1);
  }
}

// tu[k][u] = e^{-i k theta} at the first offset of unit u (zero for padding units).
__global__ void k_setup_tu(const SetupArgs a) {
  const int n = a.Kp1 * a.nup;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int k = idx / a.nup, u = idx - k * a.nup;
    float2 v = make_float2(0.f, 0.f);
    if (u < a.nu) {
      if (a.dense) {
        const double2 t = dense_twiddle(k, a.l0 + a.units[u].x, a.step, a.L);
        v = make_float2((float)t.x, (float)t.y);
      } else {
        int off = (a.l0 + a.units[u].x) % a.L;
        if (off < 0) off += a.L;
        v = a.tf32[(int)(((long long)k * off) % a.L)];
      }
    }
    a.tu[idx] = v;
  }
}

// Distance-unit table of the batch sweep: (cos t - 1, -sin t), t = 2 pi k d step / L, with
// cos t - 1 = -2 sin^2(t / 2) so that small angles keep their relative precision (FP64).
__global__ void k_setup_td(const SetupArgs a) {
  const int n = a.Kp1 * a.nd;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int k = idx / a.nd, d = idx - k * a.nd;
    // t / (2 pi): reduced exactly on the grid
    const double h = a.dense ? a.step * (double)((long long)k * d) / (double)a.L
                             : (double)(int)(((long long)k * d) % a.L) / (double)a.L;
    double sh, ch, s, c;
    sincospi(h, &sh, &ch);
    sincospi(2.0 * h, &s, &c);
    a.td[idx] = make_float2((float)(-2.0 * sh * sh), (float)(-s));
  }
}

// log rho_l = kappa cos theta_l + eta_l - log sum exp(...) over the window (one CTA, FP64),
// theta_l = 2 pi step (l0 + l) / L.
__global__ void k_setup_vm(int L, int Lw, int l0, double step, double kappa, const double* eta, double* rho64,
                           float* logrho32) {
  __shared__ double red[32];
  __shared__ double bc;
  const int tid = threadIdx.x;
  double mx = -INFINITY;
  for (int i = tid; i < Lw; i += blockDim.x) {
    const double t = kappa * cospi(2.0 * step * (double)(l0 + i) / (double)L) + eta[i];
    mx = fmax(mx, t);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmax(m, red[w]);
    bc = m;
  }
  __syncthreads();
  const double m = bc;
  double s = 0.0;
  for (int i = tid; i < Lw; i += blockDim.x) s += exp(kappa * cospi(2.0 * step * (double)(l0 + i) / (double)L) + eta[i] - m);
  s = warp_sum_d(s);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    bc = m + log(t);
  }
  __syncthreads();
  const double lz = bc;
  for (int i = tid; i < Lw; i += blockDim.x) {
    const double lr = kappa * cospi(2.0 * step * (double)(l0 + i) / (double)L) + eta[i] - lz;
    rho64[i] = exp(lr);
    logrho32[i] = (float)lr;
  }
}

struct SweepArgs {
  const float2* y;
  const int* shift;
  int N, Kp1, Q, M, L, Lw, B;
  int twp;
  int slot_bytes;  // bytes per image slot in shared memory
  int cp;          // row pitch (complex) of the c and W tiles
  int sp;          // row pitch (floats) of the s / w tile
  int off_ybuf, off_x, off_tw, off_tf, off_c, off_s, off_s64, off_w, off_wl, off_lr;
  float two_beta;
  double two_beta_d;
  const float2* x32;
  const float2* tw;
  const double2* tw64;
  const float2* tf32;
  const float* logrho32;
  double* part;  // [cols][G]
  int G;
  float* w_out;  // [N][Lw] or null
  Ctrl* ctrl;
};

// One EM sweep.  QEVEN: rows hold an even number of complex values and are
// read as float4 (two coefficients); NCOL: accumulator columns per thread.
template <bool QEVEN, int NCOL>
__global__ void __launch_bounds__(kSweepThreads, 1) k_em_sweep(const SweepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (a.ctrl->done) return;
  const bool want_ysq = (a.ctrl->iter == 0);
  constexpr int NT = kSweepThreads;
  constexpr int VEC = QEVEN ? 2 : 1;  // complex values per accumulator column
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* ybuf = smem + a.off_ybuf;
  float2* xs = reinterpret_cast<float2*>(smem + a.off_x);
  float2* tws = reinterpret_cast<float2*>(smem + a.off_tw);
  float2* tfs = reinterpret_cast<float2*>(smem + a.off_tf);
  float2* cs = reinterpret_cast<float2*>(smem + a.off_c);
  float* ss = reinterpret_cast<float*>(smem + a.off_s);
  double* ss64 = reinterpret_cast<double*>(smem + a.off_s64);
  float2* wsm = reinterpret_cast<float2*>(smem + a.off_w);
  float* wl = reinterpret_cast<float*>(smem + a.off_wl);
  float* lrs = reinterpret_cast<float*>(smem + a.off_lr);

  const int B = a.B, Kp1 = a.Kp1, Q = a.Q, L = a.L, Lw = a.Lw;
  const int ntiles = (a.N + B - 1) / B;
  const int stage_bytes = B * a.slot_bytes;
  const uint32_t img_bytes = (uint32_t)a.M * 8u;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  for (int i = tid; i < a.M; i += NT) xs[i] = a.x32[i];
  {
    const int kp4 = (Kp1 + 3) & ~3;
    for (int i = tid; i < kp4 * a.twp; i += NT) tws[i] = a.tw[i];
  }
  for (int i = tid; i < L; i += NT) tfs[i] = a.tf32[i];
  for (int i = tid; i < Lw; i += NT) lrs[i] = a.logrho32[i];
  for (int i = tid; i < kSweepWarps * Lw; i += NT) wl[i] = 0.f;
  __syncthreads();

  const int first = blockIdx.x;
  auto issue = [&](int tile, int s) {
    const int b0 = tile * B;
    const int nb = min(B, a.N - b0);
    mbar_arrive_expect_tx(&bar[s], (uint32_t)nb * img_bytes);
    unsigned char* dst = ybuf + s * stage_bytes;
    for (int b = 0; b < nb; ++b)
      bulk_g2s(dst + b * a.slot_bytes, a.y + (size_t)(b0 + b) * a.M, img_bytes, &bar[s]);
  };
  if (tid == 0) {
    if (first < ntiles) issue(first, 0);
    if (first + a.G < ntiles) issue(first + a.G, 1);
  }

  // accumulator columns owned by this thread
  const int ncols = a.M / VEC;
  int colf[NCOL], colk[NCOL];
#pragma unroll
  for (int c = 0; c < NCOL; ++c) {
    colf[c] = tid + c * NT;
    colk[c] = colf[c] < ncols ? (colf[c] * VEC) / Q : 0;
  }
  float acc[NCOL][2 * VEC];
  double acc64[NCOL][2 * VEC];
#pragma unroll
  for (int c = 0; c < NCOL; ++c)
#pragma unroll
    for (int e = 0; e < 2 * VEC; ++e) acc[c][e] = 0.f, acc64[c][e] = 0.0;
  double ll_acc = 0.0, ysq_acc = 0.0;

  // item walkers (b fastest so that lanes map to images)
  const int dB = NT % B, dK = NT / B;
  const int nlq = (Lw + 3) >> 2, nkq = (Kp1 + 3) >> 2;

  int it = 0;
  for (;; ++it) {
    const int tile = first + it * a.G;
    if (tile >= ntiles) break;
    const int s = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const bool ok = mbar_wait_bounded(&bar[s], parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(&a.ctrl->status, (int)MRA_ETIMEOUT);
        mbar_wait_bounded(&bar[s], parity);
        if (tile + a.G < ntiles) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
      }
      return;
    }
    const int b0 = tile * B;
    const int nb = min(B, a.N - b0);
    const unsigned char* yb = ybuf + s * stage_bytes;

    // ---- P1: c_jk = sum_q conj(y_jkq) x_kq, folded with e^{-i k theta_hat_j}
    {
      int b = tid % B, k = tid / B;
      float ysq_f = 0.f;
      for (int i = tid; i < B * Kp1; i += NT) {
        if (b < nb) {
          float cr = 0.f, ci = 0.f, sq = 0.f;
          const float2* yr = reinterpret_cast<const float2*>(yb + b * a.slot_bytes) + k * Q;
          const float2* xr = xs + k * Q;
          if constexpr (QEVEN) {
            const float4* y4 = reinterpret_cast<const float4*>(yr);
            const float4* x4 = reinterpret_cast<const float4*>(xr);
            if (want_ysq) {
              for (int p = 0; p < Q / 2; ++p) {
                const float4 yv = y4[p], xv = x4[p];
                cr = fmaf(yv.x, xv.x, cr); cr = fmaf(yv.y, xv.y, cr);
                ci = fmaf(yv.x, xv.y, ci); ci = fmaf(-yv.y, xv.x, ci);
                cr = fmaf(yv.z, xv.z, cr); cr = fmaf(yv.w, xv.w, cr);
                ci = fmaf(yv.z, xv.w, ci); ci = fmaf(-yv.w, xv.z, ci);
                sq = fmaf(yv.x, yv.x, sq); sq = fmaf(yv.y, yv.y, sq);
                sq = fmaf(yv.z, yv.z, sq); sq = fmaf(yv.w, yv.w, sq);
              }
            } else {
              for (int p = 0; p < Q / 2; ++p) {
                const float4 yv = y4[p], xv = x4[p];
                cr = fmaf(yv.x, xv.x, cr); cr = fmaf(yv.y, xv.y, cr);
                ci = fmaf(yv.x, xv.y, ci); ci = fmaf(-yv.y, xv.x, ci);
                cr = fmaf(yv.z, xv.z, cr); cr = fmaf(yv.w, xv.w, cr);
                ci = fmaf(yv.z, xv.w, ci); ci = fmaf(-yv.w, xv.z, ci);
              }
            }
          } else {
            for (int q = 0; q < Q; ++q) {
              const float2 yv = yr[q], xv = xr[q];
              cr = fmaf(yv.x, xv.x, cr); cr = fmaf(yv.y, xv.y, cr);
              ci = fmaf(yv.x, xv.y, ci); ci = fmaf(-yv.y, xv.x, ci);
              sq = fmaf(yv.x, yv.x, sq); sq = fmaf(yv.y, yv.y, sq);
            }
          }
          float2 c = make_float2(cr, ci);
          if (a.shift) {
            int sj = a.shift[b0 + b] % L;
            if (sj < 0) sj += L;
            c = cmul(c, tfs[(k * sj) % L]);
          }
          cs[b * a.cp + k] = c;
          ysq_f += sq;
        }
        b += dB;
        k += dK;
        if (b >= B) { b -= B; ++k; }
      }
      if (want_ysq) ysq_acc += (double)ysq_f;
    }
    __syncthreads();

    // ---- P2: s_jl = log rho_l + 2 beta Re sum_k c_jk Tw[k][l], four window offsets per item, in FP64
    // with the FP64 twiddles: this general fallback sweep has no peak-relative pass, and FP32
    // rounding of sums of size 2 beta |c| would move the weights by more than 1e-5
    {
      int b = tid % B, lq = tid / B;
      for (int i = tid; i < B * nlq; i += NT) {
        if (b < nb) {
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          const float2* cr = cs + b * a.cp;
          const double2* tcol = a.tw64 + 4 * lq;
          for (int k = 0; k < Kp1; ++k) {
            const float2 cf = cr[k];
            const double cx = (double)cf.x, cy = (double)cf.y;
            const double2 t0 = tcol[k * a.twp], t1 = tcol[k * a.twp + 1];
            const double2 t2 = tcol[k * a.twp + 2], t3 = tcol[k * a.twp + 3];
            s0 = fma(cx, t0.x, s0); s0 = fma(-cy, t0.y, s0);
            s1 = fma(cx, t1.x, s1); s1 = fma(-cy, t1.y, s1);
            s2 = fma(cx, t2.x, s2); s2 = fma(-cy, t2.y, s2);
            s3 = fma(cx, t3.x, s3); s3 = fma(-cy, t3.y, s3);
          }
          double* srow = ss64 + b * a.sp;
          const int l = 4 * lq;
          srow[l] = fma(a.two_beta_d, s0, (double)lrs[l]);
          if (l + 1 < Lw) srow[l + 1] = fma(a.two_beta_d, s1, (double)lrs[l + 1]);
          if (l + 2 < Lw) srow[l + 2] = fma(a.two_beta_d, s2, (double)lrs[l + 2]);
          if (l + 3 < Lw) srow[l + 3] = fma(a.two_beta_d, s3, (double)lrs[l + 3]);
        }
        b += dB;
        lq += dK;
        if (b >= B) { b -= B; ++lq; }
      }
    }
    __syncthreads();

    // ---- P3: normalise over the window (one warp per image)
    for (int b = warp; b < nb; b += kSweepWarps) {
      float* srow = ss + b * a.sp;
      const double* s64 = ss64 + b * a.sp;
      double m = -INFINITY;
      for (int l = lane; l < Lw; l += 32) m = fmax(m, s64[l]);
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      float z = 0.f;
      for (int l = lane; l < Lw; l += 32) {
        const float e = expf((float)(s64[l] - m));
        srow[l] = e;
        z += e;
      }
      z = warp_sum(z);
      const float inv = 1.f / z;
      float* wlw = wl + warp * Lw;
      float* wo = a.w_out ? a.w_out + (size_t)(b0 + b) * Lw : nullptr;
      for (int l = lane; l < Lw; l += 32) {
        const float w = srow[l] * inv;
        srow[l] = w;
        wlw[l] += w;
        if (wo) wo[l] = w;
      }
      if (lane == 0) ll_acc += m + (double)logf(z);
    }
    __syncthreads();

    // ---- P4: W_jk = sum_l w_jl conj(Tw[k][l]), folded with e^{+i k theta_hat_j}, four k per item
    {
      int b = tid % B, kq = tid / B;
      for (int i = tid; i < B * nkq; i += NT) {
        if (b < nb) {
          float2 w0 = make_float2(0.f, 0.f), w1 = w0, w2 = w0, w3 = w0;
          const float* srow = ss + b * a.sp;
          const int k0 = 4 * kq;
          const float2* t0 = tws + k0 * a.twp;
          const float2* t1 = t0 + a.twp;
          const float2* t2 = t1 + a.twp;
          const float2* t3 = t2 + a.twp;
          for (int l = 0; l < Lw; ++l) {
            const float w = srow[l];
            const float2 ta = t0[l], tb = t1[l], tc = t2[l], td = t3[l];
            w0.x = fmaf(w, ta.x, w0.x); w0.y = fmaf(-w, ta.y, w0.y);
            w1.x = fmaf(w, tb.x, w1.x); w1.y = fmaf(-w, tb.y, w1.y);
            w2.x = fmaf(w, tc.x, w2.x); w2.y = fmaf(-w, tc.y, w2.y);
            w3.x = fmaf(w, td.x, w3.x); w3.y = fmaf(-w, td.y, w3.y);
          }
          if (a.shift) {
            int sj = a.shift[b0 + b] % L;
            if (sj < 0) sj += L;
            w0 = cmul_conj_b(w0, tfs[(k0 * sj) % L]);
            w1 = cmul_conj_b(w1, tfs[((k0 + 1) * sj) % L]);
            w2 = cmul_conj_b(w2, tfs[((k0 + 2) * sj) % L]);
            w3 = cmul_conj_b(w3, tfs[((k0 + 3) * sj) % L]);
          }
          float2* wrow = wsm + b * a.cp;
          if (k0 < Kp1) wrow[k0] = w0;
          if (k0 + 1 < Kp1) wrow[k0 + 1] = w1;
          if (k0 + 2 < Kp1) wrow[k0 + 2] = w2;
          if (k0 + 3 < Kp1) wrow[k0 + 3] = w3;
        }
        b += dB;
        kq += dK;
        if (b >= B) { b -= B; ++kq; }
      }
    }
    __syncthreads();

    // ---- P5: num_kq += W_jk y_jkq over the tile
    for (int b = 0; b < nb; ++b) {
      const unsigned char* yimg = yb + b * a.slot_bytes;
      const float2* wrow = wsm + b * a.cp;
#pragma unroll
      for (int c = 0; c < NCOL; ++c) {
        if (colf[c] < ncols) {
          const float2 W = wrow[colk[c]];
          if constexpr (QEVEN) {
            const float4 yv = reinterpret_cast<const float4*>(yimg)[colf[c]];
            acc[c][0] = fmaf(W.x, yv.x, acc[c][0]); acc[c][0] = fmaf(-W.y, yv.y, acc[c][0]);
            acc[c][1] = fmaf(W.x, yv.y, acc[c][1]); acc[c][1] = fmaf(W.y, yv.x, acc[c][1]);
            acc[c][2] = fmaf(W.x, yv.z, acc[c][2]); acc[c][2] = fmaf(-W.y, yv.w, acc[c][2]);
            acc[c][3] = fmaf(W.x, yv.w, acc[c][3]); acc[c][3] = fmaf(W.y, yv.z, acc[c][3]);
          } else {
            const float2 yv = reinterpret_cast<const float2*>(yimg)[colf[c]];
            acc[c][0] = fmaf(W.x, yv.x, acc[c][0]); acc[c][0] = fmaf(-W.y, yv.y, acc[c][0]);
            acc[c][1] = fmaf(W.x, yv.y, acc[c][1]); acc[c][1] = fmaf(W.y, yv.x, acc[c][1]);
          }
        }
      }
    }
    if ((it & 15) == 15) {  // fold the FP32 tile sums into FP64 every 16 tiles
#pragma unroll
      for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int e = 0; e < 2 * VEC; ++e) acc64[c][e] += (double)acc[c][e], acc[c][e] = 0.f;
    }
    __syncthreads();  // every thread is done with stage s
    if (tid == 0 && tile + 2 * a.G < ntiles) issue(tile + 2 * a.G, s);
  }

  // ---- per-CTA partials, column-major [col][G]
#pragma unroll
  for (int c = 0; c < NCOL; ++c)
#pragma unroll
    for (int e = 0; e < 2 * VEC; ++e) acc64[c][e] += (double)acc[c][e];
  const int G = a.G, cta = blockIdx.x;
#pragma unroll
  for (int c = 0; c < NCOL; ++c) {
    if (colf[c] < ncols) {
      const int base = 2 * VEC * colf[c];  // first real column of this accumulator
#pragma unroll
      for (int e = 0; e < 2 * VEC; ++e) a.part[(size_t)(base + e) * G + cta] = acc64[c][e];
    }
  }
  __syncthreads();
  for (int l = tid; l < Lw; l += NT) {
    double s = 0.0;
    for (int w = 0; w < kSweepWarps; ++w) s += (double)wl[w * Lw + l];
    a.part[(size_t)(2 * a.M + l) * G + cta] = s;
  }
  __shared__ double red[2][kSweepWarps];
  ll_acc = warp_sum_d(ll_acc);
  ysq_acc = warp_sum_d(ysq_acc);
  if (lane == 0) red[0][warp] = ll_acc, red[1][warp] = ysq_acc;
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kSweepWarps; ++w) t0 += red[0][w], t1 += red[1][w];
    a.part[(size_t)(2 * a.M + Lw) * G + cta] = t0;
    a.part[(size_t)(2 * a.M + Lw + 1) * G + cta] = t1;
  }
}

}  // namespace mra

#include "update_impl.cuh"

namespace mra {

// One EM finalize in one launch: every CTA reduces its share of the columns (a warp per column, the
// fixed order of k_reduce_cols, so the totals are bit for bit the same), and the last CTA to finish
// (a ticket in the control block, taken after a fence) runs the update on the totals, which it reads
// through L2, and clears the ticket for the next launch.
__global__ void __launch_bounds__(kUpdateThreads, 1) k_finalize(const UpdateArgs a, const double* part, int G,
                                                                int cols) {
  if (__ldcg(&a.ctrl->done)) return;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int col = blockIdx.x * nw + warp; col < cols; col += gridDim.x * nw)
    reduce_cols_warp(part, G, col, const_cast<double*>(a.tot));
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&a.ctrl->fin, 1u) == gridDim.x - 1u;
    if (last) __threadfence();
  }
  __syncthreads();
  if (!last) return;
  update_body(a);
  if (threadIdx.x == 0) atomicExch(&a.ctrl->fin, 0u);
}

// tot[col] = sum_g part[col][g] in FP64, one warp per column, fixed summation order.
__global__ void k_reduce_cols(const double* part, int G, int cols, double* tot, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= cols) return;
  reduce_cols_warp(part, G, col, tot);
}

// em_run epilogue: final state out.
__global__ void k_export(int M, int Lw, const double2* x64, const double* rho64, double2* x_out, double* log_rho_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(M, Lw); i += gridDim.x * blockDim.x) {
    if (i < M) x_out[i] = x64[i];
    if (i < Lw) log_rho_out[i] = log(rho64[i]);
  }
}

struct GradArgs {
  int N, M, L, Lw, l0;
  double step;
  double sigma2, beta, kappa;
  const double* tot;
  int cols;
  const double2* x64;
  const double* rho64;
  double* loglik_out;
  double2* dx_out;
  double* dlogits_out;
  double* dkappa_out;
};

__global__ void k_grad(const GradArgs a) {
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  double nx = 0.0;
  for (int e = tid; e < a.M; e += nt) {
    const double2 x = a.x64[e];
    nx += x.x * x.x + x.y * x.y;
    if (a.dx_out)
      a.dx_out[e] = make_double2(2.0 * a.beta * (a.tot[2 * e] - a.N * x.x), 2.0 * a.beta * (a.tot[2 * e + 1] - a.N * x.y));
  }
  nx = block_sum_d(nx, red);
  double dk = 0.0;
  for (int l = tid; l < a.Lw; l += nt) {
    const double g = a.tot[2 * a.M + l] - (double)a.N * a.rho64[l];
    if (a.dlogits_out) a.dlogits_out[l] = g;
    dk += g * cospi(2.0 * a.step * (double)(a.l0 + l) / (double)a.L);
  }
  dk = block_sum_d(dk, red);
  if (tid == 0) {
    if (a.dkappa_out) *a.dkappa_out = dk;
    if (a.loglik_out)
      *a.loglik_out = a.tot[2 * a.M + a.Lw] - a.beta * a.tot[2 * a.M + a.Lw + 1] - (double)a.N * a.beta * nx -
                      (double)a.N * (double)a.M * log(kPi * a.sigma2);
  }
}

// ---- align and average: partial sums of y_j e^{+i k theta_hat_j} per CTA
template <bool QEVEN, int NCOL>
__global__ void __launch_bounds__(kSweepThreads) k_align_partial(const float2* y, const int* shift, int N, int M, int Q,
                                                                  int L, const float2* tf32, double* part, int G) {
  constexpr int VEC = QEVEN ? 2 : 1;
  const int tid = threadIdx.x, ncols = M / VEC;
  float acc[NCOL][2 * VEC];
  double acc64[NCOL][2 * VEC];
#pragma unroll
  for (int c = 0; c < NCOL; ++c)
#pragma unroll
    for (int e = 0; e < 2 * VEC; ++e) acc[c][e] = 0.f, acc64[c][e] = 0.0;
  int cnt = 0;
  for (int j = blockIdx.x; j < N; j += G) {
    int sj = shift ? shift[j] % L : 0;
    if (sj < 0) sj += L;
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
      const int f = tid + c * kSweepThreads;
      if (f < ncols) {
        const int k = (f * VEC) / Q;
        const float2 t = tf32[(k * sj) % L];  // conj(t) = e^{+i k theta_hat_j}
        if constexpr (QEVEN) {
          const float4 v = reinterpret_cast<const float4*>(y + (size_t)j * M)[f];
          acc[c][0] += v.x * t.x + v.y * t.y;
          acc[c][1] += v.y * t.x - v.x * t.y;
          acc[c][2] += v.z * t.x + v.w * t.y;
          acc[c][3] += v.w * t.x - v.z * t.y;
        } else {
          const float2 v = y[(size_t)j * M + f];
          acc[c][0] += v.x * t.x + v.y * t.y;
          acc[c][1] += v.y * t.x - v.x * t.y;
        }
      }
    }
    if (++cnt == 32) {
      cnt = 0;
#pragma unroll
      for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int e = 0; e < 2 * VEC; ++e) acc64[c][e] += (double)acc[c][e], acc[c][e] = 0.f;
    }
  }
#pragma unroll
  for (int c = 0; c < NCOL; ++c) {
    const int f = tid + c * kSweepThreads;
    if (f < ncols) {
#pragma unroll
      for (int e = 0; e < 2 * VEC; ++e) part[(size_t)(2 * VEC * f + e) * G + blockIdx.x] = acc64[c][e] + (double)acc[c][e];
    }
  }
}

__global__ void k_scale_out(int M, const double* tot, double inv, double2* x_out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x)
    x_out[e] = make_double2(tot[2 * e] * inv, tot[2 * e + 1] * inv);
}

// Algorithm 1 centring: c = argmax_s Re sum_k g_k e^{-2 pi i k s/L}, g_k = sum_q xbar_kq conj(x_kq)  (FP64, one CTA)
__global__ void k_center(int Kp1, int Q, int L, const double* tot, double invN, const double2* x_true,
                         const double2* tf64, int* center_ws, int* center_out) {
  extern __shared__ __align__(16) unsigned char csm[];
  double2* g = reinterpret_cast<double2*>(csm);
  __shared__ double rv[32];
  __shared__ int ri[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < Kp1; k += nt) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < Q; ++q) {
      const int e = k * Q + q;
      const double2 xb = make_double2(tot[2 * e] * invN, tot[2 * e + 1] * invN);
      const double2 x = x_true[e];
      s.x += xb.x * x.x + xb.y * x.y;
      s.y += xb.y * x.x - xb.x * x.y;
    }
    g[k] = s;
  }
  __syncthreads();
  double best = -INFINITY;
  int bi = 0x7fffffff;
  for (int l = tid; l < L; l += nt) {
    double s = 0.0;
    int m = 0;
    for (int k = 0; k < Kp1; ++k) {
      const double2 t = tf64[m];
      s += g[k].x * t.x - g[k].y * t.y;
      m += l;
      if (m >= L) m -= L;
    }
    if (s > best || (s == best && l < bi)) best = s, bi = l;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
  }
  if ((tid & 31) == 0) rv[tid >> 5] = best, ri[tid >> 5] = bi;
  __syncthreads();
  if (tid == 0) {
    double b = rv[0];
    int i = ri[0];
    for (int w = 1; w < (nt + 31) / 32; ++w)
      if (rv[w] > b || (rv[w] == b && ri[w] < i)) b = rv[w], i = ri[w];
    *center_ws = i;
    if (center_out) *center_out = i;
  }
}

__global__ void k_hist(int N, int L, const int* s_true, const int* s_est, const int* center, int* hist) {
  const int c = *center;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    long long r = ((long long)s_true[j] - (long long)s_est[j] + c) % L;
    if (r < 0) r += L;
    atomicAdd(hist + r, 1);
  }
}

// ============================================================================ host side
// Instances of the batch sweep that read the distance-unit table from global memory
// (sweep3_impl.cuh): batches of 8 or 4 images.
SweepV3Fn sweep_v3g_qh4(int bi, int yf);
SweepV3Fn sweep_v3g_qh8(int bi, int yf);
SweepV3Fn sweep_v3g_qh12(int bi, int yf);
SweepV3Fn sweep_v3g_qh16(int bi, int yf);

namespace {

struct SweepPlan {
  int B, slot_bytes, cp, sp, smem;
  int off_ybuf, off_x, off_tw, off_tf, off_c, off_s, off_s64, off_w, off_wl, off_lr;
};

inline int al16(int v) { return (v + 15) & ~15; }

// Shared-memory plan of the sweep: the largest tile (<= 32 images) whose two stages fit.
bool plan_sweep(int Kp1, int Q, int L, int Lw, int max_smem, SweepPlan* p) {
  const int M = Kp1 * Q;
  int slot = al16(M * 8);
  if (((slot / 16) & 1) == 0) slot += 16;  // odd number of 16-byte units: conflict-free across images
  const int cp = (Kp1 & 1) ? Kp1 : Kp1 + 1;
  const int sp = (Lw & 1) ? Lw : Lw + 1;
  const int kp4 = (Kp1 + 3) & ~3, twp = (Lw + 3) & ~3;
  for (int B = 32; B >= 1; --B) {
    int o = 128;  // two mbarriers
    p->off_ybuf = o; o += 2 * B * slot;
    p->off_x = o; o += al16(M * 8);
    p->off_tw = o; o += al16(kp4 * twp * 8);
    p->off_tf = o; o += al16(L * 8);
    p->off_c = o; o += al16(B * cp * 8);
    p->off_s = o; o += al16(B * sp * 4);
    p->off_s64 = o; o += al16(B * sp * 8);
    p->off_w = o; o += al16(B * cp * 8);
    p->off_wl = o; o += al16(kSweepWarps * Lw * 4);
    p->off_lr = o; o += al16(Lw * 4);
    if (o + 1024 <= max_smem) {  // leave room for the static reduction scratch
      p->B = B;
      p->slot_bytes = slot;
      p->cp = cp;
      p->sp = sp;
      p->smem = o;
      return true;
    }
  }
  return false;
}

struct V2Plan {
  SweepV2Launch launch;
  int nwarps, slot_bytes, sp, smem;
  int lwc;  // the warp sweep's window mode (see sweep_impl.cuh); 0 for the lean sweep
  int off_ring, off_x, off_tu, off_tf, off_lr, off_units, off_s, off_wl;
};

// Shared-memory plan of the warp-streaming sweep: each warp carries one image per stage of a
// two-stage ring; as many warps as fit, at least enough that the ring can hold every warp's
// sums at the end.
bool plan_v2(int Kp1, int Q, int L, int Lw, int nup, int max_smem, V2Plan* p) {
  if (Q % 8 != 0 || Q / 8 > 4) return false;
  const int QV = Q / 8, MR = (Kp1 + 7) / 8;
  if (MR > 7) return false;
  const int M = Kp1 * Q;
  const int slot = al16(M * 8);
  const int sp = (Lw + 3) & ~3;
  const int ipw = 1;  // two images per warp measured slower (fewer resident warps)
  const int lwc0 = nup != kUnitChunk ? 0 : Lw <= 32 ? 1 : Lw <= 64 ? 2 : 0;  // one unit chunk: fixed loops
  // a window whose unit table does not fit next to the rings reads it from global memory (lwc -1)
  for (int lwc : {lwc0, lwc0 == 0 ? -1 : lwc0}) {
    SweepV2Launch ln = QV == 1 ? sweep_v2_q1(MR, ipw, lwc) : QV == 2 ? sweep_v2_q2(MR, ipw, lwc)
                     : QV == 3 ? sweep_v2_q3(MR, ipw, lwc) : sweep_v2_q4(MR, ipw, lwc);
    if (!ln.fn) continue;
    const int maxw = ln.threads / 32;
    for (int nw = maxw; nw * 2 * ipw >= maxw && nw >= 1; --nw) {
      int o = al16(2 * maxw * 8);
      p->off_ring = o; o += 2 * ipw * nw * slot;
      p->off_x = o; o += al16(M * 8);
      p->off_tu = o; o += lwc >= 0 ? al16(Kp1 * nup * 8) : 0;
      p->off_tf = o; o += al16(L * 8);
      p->off_lr = o; o += al16(Lw * 4);
      p->off_units = o; o += al16(nup * 8);
      p->off_s = o; o += al16(maxw * ipw * sp * 4);
      p->off_wl = o; o += al16(maxw * sp * 4);
      if (o + 1024 <= max_smem) {
        p->launch = ln;
        p->nwarps = nw;
        p->slot_bytes = slot;
        p->sp = sp;
        p->smem = o;
        p->lwc = lwc;
        return true;
      }
    }
  }
  return false;
}

// Shared-memory plan of the lean warp sweep (grid windows of at most 32 mirror units that
// are not the whole circle): the warp sweep's ring and tables, and one per-warp buffer serving
// c_k (pass 1) and the window's values (images off the fast path).
bool plan_v5(int Kp1, int Q, int L, int Lw, int nu, int nup, bool dense, int max_smem, V2Plan* p, int* cbp_out) {
  if (dense || Lw >= L || nu > 32 || Q % 8 != 0 || Q / 8 > 4) return false;
  const int QV = Q / 8, MR = (Kp1 + 7) / 8;
  if (MR > 7) return false;
  const SweepV2Launch ln = QV == 1 ? sweep_v5_q1(MR, nup) : QV == 2 ? sweep_v5_q2(MR, nup)
                         : QV == 3 ? sweep_v5_q3(MR, nup) : sweep_v5_q4(MR, nup);
  if (!ln.fn) return false;
  const int M = Kp1 * Q;
  const int slot = al16(M * 8);
  const int sp = (Lw + 3) & ~3;
  const int cbp = std::max(8 * MR, (sp + 1) / 2 + 1) & ~1;  // float2: rows up to 8 MR, or Lw floats
  const int maxw = ln.threads / 32;
  for (int nw = maxw; nw * 2 >= maxw && nw >= 1; --nw) {
    int o = al16(2 * maxw * 8);
    p->off_ring = o; o += 2 * nw * slot;
    p->off_x = o; o += al16(M * 8);
    p->off_tu = o; o += al16(8 * MR * nup * 8);  // rows padded to 8 MR
    p->off_tf = o; o += al16(L * 8);
    p->off_lr = o; o += al16(Lw * 4);
    p->off_units = o; o += al16(nup * 8);
    p->off_s = o; o += al16(maxw * cbp * 8);
    p->off_wl = o; o += al16(maxw * sp * 4);
    if (o + 1024 <= max_smem) {
      p->launch = ln;
      p->nwarps = nw;
      p->slot_bytes = slot;
      p->sp = sp;
      p->smem = o;
      p->lwc = 0;
      *cbp_out = cbp;
      return true;
    }
  }
  return false;
}

// Shared-memory plan of the paired-warp sweep (grid windows of at most 32 mirror units that are
// not the whole circle, K <= 16 MR with MR x QV <= 6): per pair a ring of three image slots
// (two where three do not fit), the unit table in row pairs, the grid twiddles and the small
// per-warp and per-pair exchange buffers.
struct V6Plan {
  SweepV6Launch launch;
  int ns, slot_bytes, sp, smem;
  int off_bar, off_ring, off_tab, off_tf, off_lr, off_units, off_cb, off_xp, off_xq, off_pv, off_sb, off_wl;
};
bool plan_v6(int Kp1, int Q, int L, int Lw, int nu, bool dense, int max_smem, V6Plan* p) {
  const int K = Kp1 - 1;
  if (dense || Lw >= L || nu > 32 || K < 1 || L > 100000 || Q % 8 != 0 || Q / 8 > 4) return false;
  const int QV = Q / 8, MR = (K + 15) / 16;
  if (MR * QV > 6) return false;
  const SweepV6Launch ln = QV == 1 ? sweep_v6_q1(MR) : QV == 2 ? sweep_v6_q2(MR)
                         : QV == 3 ? sweep_v6_q3(MR) : sweep_v6_q4(MR);
  if (!ln.fn) return false;
  const int NW = ln.threads / 32, NP = NW / 2;
  const int M = Kp1 * Q;
  const int slot = al16(M * 8);
  const int sp = (Lw + 3) & ~3;
  for (int ns = 3; ns >= 2; --ns) {
    int o = 0;
    p->off_bar = o; o += al16(NP * ns * 8);
    p->off_ring = o; o += NP * ns * slot;
    p->off_tab = o; o += 8 * MR * 32 * 16;
    p->off_tf = o; o += al16(L * 8);
    p->off_lr = o; o += al16(Lw * 4);
    p->off_units = o; o += 32 * 8;
    p->off_cb = o; o += NW * 8 * MR * 8;
    p->off_xp = o; o += NP * 64 * 8;
    p->off_xq = o; o += NP * 8 * 8;
    p->off_pv = o; o += al16(NP * 2 * sp * 4);
    p->off_sb = o; o += al16(NW * sp * 4);
    p->off_wl = o; o += al16(NP * sp * 4);
    if (o + 1024 <= max_smem) {
      p->launch = ln;
      p->ns = ns;
      p->slot_bytes = slot;
      p->sp = sp;
      p->smem = o;
      return true;
    }
  }
  return false;
}

// Plan of the split sweep: the stream kernels' ring (two slots per warp), x and
// the grid twiddles; the transform kernel's B operand, two A tiles, tables and reduction scratch
// (at least 116 KB, so that one transform CTA holds a streaming multiprocessor's tensor memory).
struct SplitPlan {
  SplitStreamFns fns;
  SplitTransFn trans;
  int KP, KA, NP, ncols, smem1, smem2, nwarps, slot_bytes;
  int off_ring, off_x, off_tf;
  int k2_off_b, k2_off_ah, k2_off_al, k2_off_lr, k2_off_tf, k2_off_wt, k2_off_ll, k2_off_cs, k2_off_td;
  int k2_off_info;
  int k2_ndp;
};
bool plan_split(int Kp1, int Q, int L, int Lw, int max_smem, SplitPlan* p) {
  if (!split_possible(Kp1, Q, Lw)) return false;
  const int QV = Q / 8, MR = (Kp1 + 7) / 8;
  if (MR > 6) return false;
  p->fns = QV == 1 ? sweep_tc_q1(MR) : QV == 2 ? sweep_tc_q2(MR) : QV == 3 ? sweep_tc_q3(MR) : sweep_tc_q4(MR);
  p->KP = (Kp1 + 3) / 4 * 4;
  p->trans = sweep_tc_trans(p->KP);
  if (!p->fns.corr || !p->trans) return false;
  p->KA = (2 * p->KP + 15) / 16 * 16;
  p->NP = (Lw + 15) / 16 * 16;
  p->ncols = 32;  // tensor-memory columns: the window's, at most 512 (wider windows take two passes)
  while (p->ncols < p->NP && p->ncols < 512) p->ncols *= 2;
  const int M = Kp1 * Q;
  p->slot_bytes = al16(M * 8);
  const int maxw = kTcStreamThreads / 32;
  bool ok = false;
  for (int nw = maxw; nw >= maxw / 2; --nw) {
    int o = al16(2 * maxw * 8);
    p->off_ring = o; o += 2 * nw * p->slot_bytes;
    p->off_x = o; o += al16(M * 8);
    p->off_tf = o; o += al16(L * 8);
    if (o + 1024 <= max_smem) {
      p->nwarps = nw;
      p->smem1 = o;
      ok = true;
      break;
    }
  }
  if (!ok) return false;
  int o = 128;  // mbarrier and tensor-memory address
  p->k2_off_b = o; o += al16(p->NP * p->KA * 2);
  p->k2_off_ah = o; o += al16(kTcTile * p->KA * 2);
  p->k2_off_al = o; o += al16(kTcTile * p->KA * 2);
  p->k2_off_lr = o; o += al16(Lw * 4);
  p->k2_off_tf = o; o += al16(L * 8);
  o = (o + 7) & ~7;
  p->k2_off_wt = o; o += al16(Lw * 8);
  p->k2_off_ll = o; o += al16(kTcTransThreads * 8);
  p->k2_off_cs = o; o += al16(std::max(kTcTile * Kp1, kTcTransThreads) * 8);  // later the CTA's ll sums
  p->k2_off_info = o; o += al16(kTcTile * 4 * 14);  // [4][128] maxima, indices, distances; scales; bounds
  if (o + 1024 > max_smem) return false;
  // the distance-unit table in shared memory, [d][KP + 1]: whole, or its first distances (those near
  // each image's peak, where pass 2 works) with the rest read from global memory
  const int nd = Lw == L ? L / 2 + 1 : Lw;
  const int ndp = std::min(nd, std::max(0, (max_smem - 1024 - o) & ~15) / ((p->KP + 1) * 8));
  if (ndp >= 8) {
    p->k2_off_td = o;
    p->k2_ndp = ndp;
    o += al16((p->KP + 1) * ndp * 8);
  } else {
    p->k2_off_td = 0;
    p->k2_ndp = 0;
  }
  p->smem2 = std::max(o, 116 * 1024);
  return p->smem2 + 1024 <= max_smem;
}

struct V3Plan {
  SweepV3Fn fn;
  int bi, ns, slot_bytes, cp, sp, dp, nd, wrap, r0, d1, phase0, fsplit, smem;
  int tdg;  // 1: the distance-unit table stays in global memory
  int off_ring, off_x, off_xr, off_td, off_tf, off_lr, off_c, off_s, off_w2, off_info, off_wl;
};

// Shared-memory plan of the CTA-cooperative sweep: the first (batch, stages) of
// (16, 2), (12, 2), (8, 3), (8, 2), (4, 3), (4, 2) whose ring and tables fit; failing that
// (a wide dense window), the first of (8, 3), (8, 2), (4, 3), (4, 2) that fits with the
// distance-unit table left in global memory (tdg, forced by force_tdg).  Per-image pitches
// are odd (in words of their element type) so that the images of one warp fall in
// distinct banks.
bool plan_v3(int Kp1, int Q, int L, int Lw, int l0, bool dense, int yf, int want_bi, int want_ns, int max_smem,
             V3Plan* p, bool force_tdg = false) {
  if (Q % 8 != 0) return false;
  const int QH = Q / 2;
  if (Kp1 * (QH / 2) > kV3Threads) return false;
  const int M = Kp1 * Q;
  int words = (M * 8 + 15) / 16;
  if (words % 2 == 0) ++words;
  const int slot = words * 16;
  p->wrap = !dense && Lw == L ? 1 : 0;
  p->nd = p->wrap ? L / 2 + 1 : Lw;
  int r0 = dense ? -l0 : (-l0) % L;  // the window index of rotation 0
  if (r0 < 0) r0 += dense ? Lw : L;
  if (r0 >= Lw || r0 < 0) r0 = Lw / 2;  // rotation 0 outside the window: start from its centre
  p->r0 = r0;
  p->d1 = p->wrap ? L / 2 : std::max(r0, Lw - 1 - r0);
  p->phase0 = dense ? 0 : ((l0 + r0) % L + L) % L;
  const int cp = Kp1 | 1, sp = Lw | 1, dp = p->nd | 1;
  const int cfg[6][2] = {{16, 2}, {12, 2}, {8, 3}, {8, 2}, {4, 3}, {4, 2}};
  for (int tdg = force_tdg ? 1 : 0; tdg < 2; ++tdg) {
    for (const auto& bn : cfg) {
      const int bi = bn[0], ns = bn[1];
      if ((want_bi && bi != want_bi) || (want_ns && ns != want_ns)) continue;
      const SweepV3Fn fn = tdg ? (QH == 4 ? sweep_v3g_qh4(bi, yf) : QH == 8 ? sweep_v3g_qh8(bi, yf)
                                 : QH == 12 ? sweep_v3g_qh12(bi, yf) : QH == 16 ? sweep_v3g_qh16(bi, yf) : nullptr)
                               : (QH == 4 ? sweep_v3_qh4(bi, yf) : QH == 8 ? sweep_v3_qh8(bi, yf)
                                 : QH == 12 ? sweep_v3_qh12(bi, yf) : QH == 16 ? sweep_v3_qh16(bi, yf) : nullptr);
      if (!fn) {
        if (tdg) continue;  // no global-table instance for this batch
        return false;        // no instance for this row width
      }
      int o = 128;  // ring mbarriers
      p->off_ring = o; o += ns * bi * slot;
      p->off_x = o; o += al16(M * 8);
      p->off_xr = o; o += al16(M * 8);
      p->off_td = o; o += tdg ? 0 : al16(Kp1 * dp * 8);
      p->off_tf = o; o += al16(L * 8);
      p->off_lr = o; o += al16(Lw * 4);
      p->off_c = o; o += al16(bi * cp * 8);
      p->off_s = o; o += al16(bi * sp * 4);
      p->off_w2 = o; o += al16(bi * dp * 8);
      p->off_info = o; o += al16(bi * 16);
      p->off_wl = o; o += al16((kV3Threads / 32) * sp * 4);
      if (o + 1024 <= max_smem) {
        p->fn = fn;
        p->bi = bi;
        p->ns = ns;
        p->slot_bytes = slot;
        p->cp = cp; p->sp = sp; p->dp = dp;
        p->fsplit = (p->d1 + 1) * bi * 2 <= kV3Threads ? 2 : 1;  // two threads per forward item if all fit
        p->smem = o;
        p->tdg = tdg;
        return true;
      }
    }
  }
  return false;
}

struct V4Plan {
  SweepV4Launch launch;
  int lc, slot_bytes, cp, sp, dp, nd, wrap, r0, d1, phase0, smem, grid;
  int off_ring, off_x, off_td, off_tf, off_lr, off_c, off_s, off_w2, off_info, off_wl;
};

// Shared-memory plan of the chunked two-read sweep for one launch shape: one slot per
// warp and the largest chunk of 128, 64, 32 or 16 images (or want_c) whose transform
// buffers fit in max_smem.
bool plan_v4_shape(int Kp1, int Q, int L, int Lw, int l0, bool dense, int want_c, int max_smem,
                   const SweepV4Launch& ln, V4Plan* p) {
  const int NW = ln.threads / 32;
  const int M = Kp1 * Q;
  const int slot = al16(M * 8);
  p->wrap = !dense && Lw == L ? 1 : 0;
  p->nd = p->wrap ? L / 2 + 1 : Lw;
  int r0 = dense ? -l0 : (-l0) % L;  // the window index of rotation 0
  if (r0 < 0) r0 += dense ? Lw : L;
  if (r0 >= Lw || r0 < 0) r0 = Lw / 2;
  p->r0 = r0;
  p->d1 = p->wrap ? L / 2 : std::max(r0, Lw - 1 - r0);
  p->phase0 = dense ? 0 : ((l0 + r0) % L + L) % L;
  const int cp = Kp1 | 1, sp = Lw | 1, dp = p->nd | 1;
  for (int lc = 7; lc >= 4; --lc) {
    const int c = 1 << lc;
    if ((want_c && c != want_c) || c > ln.threads) continue;
    int o = 128;  // mbarriers, one per warp
    p->off_ring = o; o += NW * slot;
    p->off_x = o; o += al16(M * 8);
    p->off_td = o; o += al16(Kp1 * dp * 8);
    p->off_tf = o; o += al16(L * 8);
    p->off_lr = o; o += al16(Lw * 4);
    p->off_c = o; o += al16(c * cp * 8);
    p->off_s = o; o += al16(c * sp * 4);
    p->off_w2 = o; o += al16(c * dp * 8);
    p->off_info = o; o += al16(c * 16);
    p->off_wl = o; o += al16(4 * NW * sp * 4);
    if (o + 1024 <= max_smem) {
      p->launch = ln;
      p->lc = lc;
      p->slot_bytes = slot;
      p->cp = cp; p->sp = sp; p->dp = dp;
      p->smem = o;
      return true;
    }
  }
  return false;
}

// Two CTAs per SM (each with half the shared memory, so that one can stream while the
// other transforms) where the plan fits, else one; want_cpsm fixes the choice.
bool plan_v4(int Kp1, int Q, int L, int Lw, int l0, bool dense, int yf, int want_c, int want_cpsm,
             const DevInfo& di, V4Plan* p) {
  if (Q % 8 != 0 || Q / 8 > 4) return false;
  const int QV = Q / 8, MR = (Kp1 + 7) / 8;
  if (MR > 7) return false;
  for (int cpsm = kMaxCtasPerSm; cpsm >= 1; --cpsm) {
    if (want_cpsm && cpsm != want_cpsm) continue;
    const SweepV4Launch ln =
        yf ? (QV == 1 ? sweep_v4_q1_f1(MR, cpsm) : QV == 2 ? sweep_v4_q2_f1(MR, cpsm)
              : QV == 3 ? sweep_v4_q3_f1(MR, cpsm) : sweep_v4_q4_f1(MR, cpsm))
           : (QV == 1 ? sweep_v4_q1_f0(MR, cpsm) : QV == 2 ? sweep_v4_q2_f0(MR, cpsm)
              : QV == 3 ? sweep_v4_q3_f0(MR, cpsm) : sweep_v4_q4_f0(MR, cpsm));
    if (!ln.fn) continue;
    const int max_smem = std::min(di.max_smem_optin, di.smem_per_sm / cpsm - 1024);
    if (plan_v4_shape(Kp1, Q, L, Lw, l0, dense, want_c, max_smem, ln, p)) {
      p->grid = di.sms * cpsm;
      return true;
    }
  }
  return false;
}

// Which EM sweep a call uses.  kind: 0 = automatic, 1 = warp per image, 2 = batch
// (CTA-cooperative) with batch bi and ring stages ns (0 = the first that fits),
// 3 = chunked two-read with bi images per chunk and ns CTAs per SM (0 = first that fits),
// 4 = lean warp per image, 5 = split (tensor-core transform), 6 = paired warps per image.
struct SweepSel {
  int kind, bi, ns;
};

// MRA_SWEEP=warp|cta|chunk|lean|tc|pair, MRA_SWEEP_BI=16|12|8|4 and MRA_SWEEP_NS=2|3 fix the sweep (for
// comparisons and tuning runs); they take precedence over the autotuner's cache.
// MRA_SWEEP_TDG=1 makes the batch sweep read its distance-unit table from global memory
// even where the table fits in shared memory (to test that variant on small windows).
SweepSel env_sweep() {
  SweepSel e{0, 0, 0};
  const char* k = getenv("MRA_SWEEP");
  if (k && strcmp(k, "warp") == 0) e.kind = 1;
  if (k && strcmp(k, "cta") == 0) e.kind = 2;
  if (k && strcmp(k, "chunk") == 0) e.kind = 3;
  if (k && strcmp(k, "lean") == 0) e.kind = 4;
  if (k && strcmp(k, "tc") == 0) e.kind = 5;
  if (k && strcmp(k, "pair") == 0) e.kind = 6;
  const char* b = getenv("MRA_SWEEP_BI");
  const char* n = getenv("MRA_SWEEP_NS");
  e.bi = b ? atoi(b) : 0;
  e.ns = n ? atoi(n) : 0;
  return e;
}

bool env_tdg() {
  const char* t = getenv("MRA_SWEEP_TDG");
  return t && atoi(t) != 0;
}

// ---- autotuner cache: the fastest sweep measured for a problem shape on a device
struct TuneKey {
  int dev, Kp1, Q, L, Lw, l0, yfmt;
  double step;
  bool operator<(const TuneKey& o) const {
    const int a[7] = {dev, Kp1, Q, L, Lw, l0, yfmt}, b[7] = {o.dev, o.Kp1, o.Q, o.L, o.Lw, o.l0, o.yfmt};
    if (std::lexicographical_compare(a, a + 7, b, b + 7)) return true;
    if (std::lexicographical_compare(b, b + 7, a, a + 7)) return false;
    return step < o.step;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, SweepSel> g_tune;

TuneKey tune_key(const mra_dims* d, int Lw, int l0, double step, int yfmt) {
  int dev = 0;
  cudaGetDevice(&dev);
  return TuneKey{dev, d->K + 1, d->Q, d->L, Lw, l0, yfmt, step};
}
bool tune_lookup(const TuneKey& k, SweepSel* out) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}
void tune_store(const TuneKey& k, const SweepSel& v) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[k] = v;
}

typedef void (*SweepFn)(const SweepArgs);

SweepFn pick_sweep(bool qeven, int ncolmax) {
  if (qeven) {
    if (ncolmax <= 1) return k_em_sweep<true, 1>;
    if (ncolmax <= 2) return k_em_sweep<true, 2>;
    if (ncolmax <= 4) return k_em_sweep<true, 4>;
    if (ncolmax <= 8) return k_em_sweep<true, 8>;
    return nullptr;
  }
  if (ncolmax <= 1) return k_em_sweep<false, 1>;
  if (ncolmax <= 2) return k_em_sweep<false, 2>;
  if (ncolmax <= 4) return k_em_sweep<false, 4>;
  if (ncolmax <= 8) return k_em_sweep<false, 8>;
  return nullptr;
}

bool ptr_ok(const void* p, size_t align) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) % align) == 0; }

int check_dims(const mra_dims* d) {
  if (!d) return MRA_EINVAL;
  if (d->N < 1 || d->K < 0 || d->Q < 1 || d->L < 1) return MRA_EINVAL;
  if (!(d->sigma2 > 0.0) || !isfinite(d->sigma2)) return MRA_EINVAL;
  const long long M = (long long)(d->K + 1) * d->Q;
  if (M % 2 != 0 || M > 4096) return MRA_EINVAL;
  if ((long long)d->N * M > (1ll << 40)) return MRA_EINVAL;
  return MRA_OK;
}

// Everything one EM-type call needs on the host.
struct EmCall {
  EmLayout lay;
  SweepPlan plan;
  SweepFn sweep;
  SweepArgs sa;
  SetupArgs su;
  UpdateArgs ua;
  Ctrl* ctrl;
  double* tot;
  int reduce_blocks;
  int fin_blocks;  // CTAs of k_finalize
  int update_smem;
  bool v2;  // warp-per-image sweep (rows of Q a multiple of 8) instead of the tile sweep
  bool v5;  // with v2: the lean warp sweep's kernel and plan
  int v5_cbp;
  bool v6;  // with v2 (whose tables it reads): the paired-warp sweep
  V6Plan v6p;
  SweepV6Args sa6;
  V2Plan v2p;
  SweepV2Args sa2;
  bool v3;  // CTA-cooperative sweep over image batches
  V3Plan v3p;
  SweepV3Args sa3;
  bool v4;  // chunked two-read sweep
  V4Plan v4p;
  SweepV4Args sa4;
  bool vs;  // split sweep (tensor-core transform)
  SplitPlan sp;
  SplitArgs sa5;
  void set_w_out(float* w) {
    sa.w_out = w;
    sa2.w_out = w;
    sa6.w_out = w;
    sa3.w_out = w;
    sa4.w_out = w;
    sa5.w_out = w;
  }
};

// yfmt: 0 = y in complex64, 1 = y as the BF16 hi/lo split (batch sweep only).
// force: a fixed sweep (the autotuner's candidates); otherwise the environment, then the
// autotuner's cache, then the default rule below.
// step: spacing of the window's rotations in grid units (1 = the grid, see window_ok).
// smem_cap > 0: plan the sweeps for at most that much dynamic shared memory per CTA.
int prepare(const mra_dims* d, int Lw, int l0, double step, const float* y, const int32_t* shift, void* ws,
            size_t ws_bytes, EmCall* c, bool allow_v3 = true, int yfmt = 0, const SweepSel* force = nullptr,
            int smem_cap = 0) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if (!window_ok(d->L, Lw, l0, step)) return MRA_EINVAL;
  const bool dense = step != 1.0;
  if (!ptr_ok(y, 16) || !ptr_ok(ws, 256)) return MRA_EINVAL;
  if (shift && !ptr_ok(shift, 4)) return MRA_EINVAL;
  DevInfo di;
  if ((st = dev_info(&di)) != MRA_OK) return st;
  if (smem_cap > 0) di.max_smem_optin = std::min(di.max_smem_optin, smem_cap);
  const int G = di.sms;
  // partial sums have room for kMaxCtasPerSm CTAs per SM; lay.G is the launch grid
  c->lay = em_layout(d->N, d->K, d->Q, d->L, Lw, G * kMaxCtasPerSm);
  c->lay.G = G;
  if (ws_bytes < c->lay.total) return MRA_EWORKSPACE;
  const int Kp1 = d->K + 1, M = Kp1 * d->Q;
  const int nu = window_units(d->L, Lw, l0, dense, nullptr);
  const int nup = round_up(nu, kUnitChunk);
  SweepSel sel = env_sweep();
  if (force) {
    sel = *force;
  } else if (sel.kind == 0 && sel.bi == 0 && sel.ns == 0) {
    SweepSel tuned;
    if (tune_lookup(tune_key(d, Lw, l0, step, yfmt), &tuned)) sel = tuned;
  }
  c->v4 = false;
  c->v5 = false;
  c->v6 = false;
  c->vs = false;
  if (yfmt) {  // the batch sweep reads the split format, and the chunked sweep when chosen
    c->v2 = false;
    if (sel.kind == 3) {
      c->v3 = false;
      c->v4 = plan_v4(Kp1, d->Q, d->L, Lw, l0, dense, 1, sel.bi, sel.ns, di, &c->v4p);
      if (c->v4) c->lay.G = c->v4p.grid;
    } else {
      c->v3 = sel.kind != 1 &&
              plan_v3(Kp1, d->Q, d->L, Lw, l0, dense, 1, sel.bi, sel.ns, di.max_smem_optin, &c->v3p, env_tdg());
    }
    if (!c->v3 && !c->v4) return MRA_EINVAL;  // no sweep for this shape reads the split format
  } else {
    // By default the warp sweep keeps a window of one unit chunk in registers and is the
    // faster one there; wider windows (up to the whole circle) go to the batch sweep, unless
    // its distance-unit table would have to stay in global memory (the 721-rotation dense
    // window at |k| <= 32: 4.04 ms per sweep against 3.20 ms for the warp sweep).
    c->v5 = false;
    c->v2 = sel.kind != 2 && plan_v2(Kp1, d->Q, d->L, Lw, nup, di.max_smem_optin, &c->v2p);
    c->v3 = allow_v3 && sel.kind != 1 && (!c->v2 || sel.kind == 2 || nup > kUnitChunk) &&
            plan_v3(Kp1, d->Q, d->L, Lw, l0, dense, 0, sel.bi, sel.ns, di.max_smem_optin, &c->v3p, env_tdg());
    if (c->v3 && c->v3p.tdg && c->v2 && sel.kind != 2) c->v3 = false;
    if (c->v3) c->v2 = false;
    // The chunked two-read sweep runs when chosen (environment or autotuner): it leads on
    // sharp posteriors and ties the warp sweep on broad ones.
    if (allow_v3 && sel.kind == 3) {
      c->v4 = plan_v4(Kp1, d->Q, d->L, Lw, l0, dense, 0, sel.bi, sel.ns, di, &c->v4p);
      if (c->v4) {
        c->v2 = c->v3 = false;
        c->lay.G = c->v4p.grid;
      }
    }
    // The lean warp sweep (EM calls only; align mode stays in the warp sweep) where it plans, when
    // chosen or by default in place of the warp sweep.
    c->v5 = false;
    if (allow_v3 && (sel.kind == 4 || (sel.kind == 0 && !c->v3 && !c->v4))) {
      V2Plan p5;
      if (plan_v5(Kp1, d->Q, d->L, Lw, nu, nup, dense, di.max_smem_optin, &p5, &c->v5_cbp)) {
        c->v2p = p5;
        c->v2 = c->v5 = true;
        c->v3 = c->v4 = false;
        c->lay.G = G;
      }
    }
    // The paired-warp sweep (EM calls only) where it plans, when chosen (it ties the lean sweep at the
    // benchmark's shape: 0.225 ms per sweep).
    c->v6 = false;
    if (allow_v3 && sel.kind == 6 &&
        plan_v6(Kp1, d->Q, d->L, Lw, nu, dense, di.max_smem_optin, &c->v6p)) {
      c->v2 = c->v6 = true;  // v2: the warp sweep's tables
      c->v3 = c->v4 = c->v5 = false;
      c->lay.G = G;
    }
    // The split sweep (tensor-core transform) for windows wider than 64 rotations when chosen, and by
    // default for the whole circle (full search: 0.45 ms against the batch sweep's 0.73 ms per step at
    // |k| <= 32, Q = 24, N = 1e5, L = 360 on sharp posteriors).
    c->vs = false;
    const bool split_default = sel.kind == 0 && !dense && Lw == d->L && Lw <= 512;
    if (allow_v3 && (sel.kind == 5 || split_default) && split_possible(Kp1, d->Q, Lw) &&
        plan_split(Kp1, d->Q, d->L, Lw, di.max_smem_optin, &c->sp)) {
      c->vs = true;
      c->v2 = c->v3 = c->v4 = c->v5 = c->v6 = false;
      c->lay.G = G;
    }
    if (force && ((force->kind == 1 && !c->v2) || (force->kind == 2 && !c->v3) || (force->kind == 3 && !c->v4) ||
                  (force->kind == 4 && !c->v5) || (force->kind == 5 && !c->vs) || (force->kind == 6 && !c->v6)))
      return MRA_EINVAL;
  }
  if (c->vs) {
    if (raise_smem_limit(reinterpret_cast<const void*>(c->sp.fns.corr), c->sp.smem1) != MRA_OK ||
        raise_smem_limit(reinterpret_cast<const void*>(c->sp.fns.accum), c->sp.smem1) != MRA_OK ||
        raise_smem_limit(reinterpret_cast<const void*>(c->sp.trans), c->sp.smem2) != MRA_OK)
      return MRA_ECUDA;
    c->sweep = nullptr;
  } else if (c->v4) {
    if (raise_smem_limit(reinterpret_cast<const void*>(c->v4p.launch.fn), c->v4p.smem) != MRA_OK) return MRA_ECUDA;
    c->sweep = nullptr;
  } else if (c->v3) {
    if (raise_smem_limit(reinterpret_cast<const void*>(c->v3p.fn), c->v3p.smem) != MRA_OK)
      return MRA_ECUDA;
    c->sweep = nullptr;
  } else if (c->v6) {
    if (raise_smem_limit(reinterpret_cast<const void*>(c->v6p.launch.fn), c->v6p.smem) != MRA_OK)
      return MRA_ECUDA;
    c->sweep = nullptr;
  } else if (c->v2) {
    if (raise_smem_limit(reinterpret_cast<const void*>(c->v2p.launch.fn), c->v2p.smem) != MRA_OK)
      return MRA_ECUDA;
    c->sweep = nullptr;
  } else {
    if (!plan_sweep(Kp1, d->Q, d->L, Lw, di.max_smem_optin, &c->plan)) return MRA_EINVAL;
    const bool qeven = (d->Q % 2) == 0;
    const int vec = qeven ? 2 : 1;
    const int ncolmax = (M / vec + kSweepThreads - 1) / kSweepThreads;
    c->sweep = pick_sweep(qeven, ncolmax);
    if (!c->sweep) return MRA_EINVAL;
    if (raise_smem_limit(reinterpret_cast<const void*>(c->sweep), c->plan.smem) != MRA_OK)
      return MRA_ECUDA;
  }
  unsigned char* base = static_cast<unsigned char*>(ws);
  const EmLayout& L_ = c->lay;
  c->ctrl = reinterpret_cast<Ctrl*>(base + L_.ctrl);
  c->tot = reinterpret_cast<double*>(base + L_.tot);

  SweepArgs& s = c->sa;
  s.y = reinterpret_cast<const float2*>(y);
  s.shift = shift;
  s.N = d->N; s.Kp1 = Kp1; s.Q = d->Q; s.M = M; s.L = d->L; s.Lw = Lw; s.B = c->plan.B;
  s.twp = L_.twp;
  s.slot_bytes = c->plan.slot_bytes; s.cp = c->plan.cp; s.sp = c->plan.sp;
  s.off_ybuf = c->plan.off_ybuf; s.off_x = c->plan.off_x; s.off_tw = c->plan.off_tw; s.off_tf = c->plan.off_tf;
  s.off_c = c->plan.off_c; s.off_s = c->plan.off_s; s.off_s64 = c->plan.off_s64; s.off_w = c->plan.off_w; s.off_wl = c->plan.off_wl;
  s.off_lr = c->plan.off_lr;
  s.two_beta = (float)(2.0 / d->sigma2);
  s.two_beta_d = 2.0 / d->sigma2;
  s.x32 = reinterpret_cast<const float2*>(base + L_.x32);
  s.tw = reinterpret_cast<const float2*>(base + L_.tw);
  s.tw64 = reinterpret_cast<const double2*>(base + L_.tw64);
  s.tf32 = reinterpret_cast<const float2*>(base + L_.tf32);
  s.logrho32 = reinterpret_cast<const float*>(base + L_.logrho32);
  s.part = reinterpret_cast<double*>(base + L_.part);
  s.G = G;
  s.w_out = nullptr;
  s.ctrl = c->ctrl;

  SweepV2Args& v = c->sa2;
  v.y = s.y;
  v.shift = shift;
  v.N = d->N; v.Kp1 = Kp1; v.M = M; v.L = d->L; v.Lw = Lw; v.NU = nu; v.NUP = nup;
  v.nwarps = c->v2p.nwarps; v.slot_bytes = c->v2p.slot_bytes; v.sp = c->v2p.sp;
  v.off_ring = c->v2p.off_ring; v.off_x = c->v2p.off_x; v.off_tu = c->v2p.off_tu; v.off_tf = c->v2p.off_tf;
  v.off_lr = c->v2p.off_lr; v.off_units = c->v2p.off_units; v.off_s = c->v2p.off_s; v.off_wl = c->v2p.off_wl;
  v.cbp = c->v5 ? c->v5_cbp : 0;
  v.two_beta = s.two_beta;
  v.align_only = 0;
  v.wrap = !dense && Lw == d->L ? 1 : 0;
  v.l0m = ((l0 % d->L) + d->L) % d->L;
  v.nd = v.wrap ? d->L / 2 + 1 : Lw;
  v.td = reinterpret_cast<const float2*>(base + L_.td);
  v.tw = dense ? s.tw : nullptr;
  v.twp = L_.twp;
  v.x32 = s.x32;
  v.tu = reinterpret_cast<const float2*>(base + L_.tu);
  v.units = reinterpret_cast<const int2*>(base + L_.units);
  v.tf32 = s.tf32;
  v.logrho32 = s.logrho32;
  v.part = s.part;
  v.G = G;
  v.w_out = nullptr;
  v.ctrl = c->ctrl;

  SweepV6Args& v6 = c->sa6;
  const V6Plan& q6 = c->v6p;
  v6.y = s.y;
  v6.shift = shift;
  v6.N = d->N; v6.K = d->K; v6.M = M; v6.L = d->L; v6.Lw = Lw; v6.NU = nu;
  v6.ns = q6.ns; v6.slot_bytes = q6.slot_bytes; v6.sp = q6.sp;
  v6.off_bar = q6.off_bar; v6.off_ring = q6.off_ring; v6.off_tab = q6.off_tab; v6.off_tf = q6.off_tf;
  v6.off_lr = q6.off_lr; v6.off_units = q6.off_units; v6.off_cb = q6.off_cb; v6.off_xp = q6.off_xp;
  v6.off_xq = q6.off_xq; v6.off_pv = q6.off_pv; v6.off_sb = q6.off_sb; v6.off_wl = q6.off_wl;
  v6.two_beta = s.two_beta;
  v6.l0m = v.l0m;
  v6.nd = v.nd;
  v6.nup = nup;
  v6.x32 = s.x32;
  v6.tu = v.tu;
  v6.units = v.units;
  v6.td = v.td;
  v6.tf32 = s.tf32;
  v6.logrho32 = s.logrho32;
  v6.part = s.part;
  v6.G = G;
  v6.w_out = nullptr;
  v6.ctrl = c->ctrl;

  SweepV3Args& w = c->sa3;
  const V3Plan& q3 = c->v3p;
  w.y = s.y;
  w.shift = shift;
  w.N = d->N; w.Kp1 = Kp1; w.M = M; w.L = d->L; w.Lw = Lw;
  w.ns = q3.ns; w.slot_bytes = q3.slot_bytes; w.cp = q3.cp; w.sp = q3.sp; w.dp = q3.dp; w.nd = q3.nd;
  w.wrap = q3.wrap; w.r0 = q3.r0; w.d1 = q3.d1; w.phase0 = q3.phase0; w.fsplit = q3.fsplit;
  w.off_ring = q3.off_ring; w.off_x = q3.off_x; w.off_xr = q3.off_xr; w.off_td = q3.off_td; w.off_tf = q3.off_tf;
  w.off_lr = q3.off_lr; w.off_c = q3.off_c; w.off_s = q3.off_s; w.off_w2 = q3.off_w2; w.off_info = q3.off_info;
  w.off_wl = q3.off_wl;
  w.two_beta = s.two_beta;
  w.two_beta_d = 2.0 / d->sigma2;
  w.x32 = s.x32;
  w.td = reinterpret_cast<const float2*>(base + L_.td);
  w.tf32 = s.tf32;
  w.tw = dense ? s.tw : nullptr;
  w.twp = L_.twp;
  w.logrho32 = s.logrho32;
  w.part = s.part;
  w.w_out = nullptr;
  w.ctrl = c->ctrl;

  SweepV4Args& v4 = c->sa4;
  const V4Plan& q4 = c->v4p;
  v4.y = s.y;
  v4.shift = shift;
  v4.N = d->N; v4.Kp1 = Kp1; v4.M = M; v4.L = d->L; v4.Lw = Lw;
  v4.slot_bytes = q4.slot_bytes; v4.cp = q4.cp; v4.sp = q4.sp; v4.dp = q4.dp;
  v4.nd = q4.nd; v4.wrap = q4.wrap; v4.r0 = q4.r0; v4.d1 = q4.d1; v4.phase0 = q4.phase0; v4.lc = q4.lc;
  v4.off_ring = q4.off_ring; v4.off_x = q4.off_x; v4.off_td = q4.off_td; v4.off_tf = q4.off_tf;
  v4.off_lr = q4.off_lr; v4.off_c = q4.off_c; v4.off_s = q4.off_s; v4.off_w2 = q4.off_w2;
  v4.off_info = q4.off_info; v4.off_wl = q4.off_wl;
  v4.two_beta = s.two_beta;
  v4.x32 = s.x32;
  v4.td = reinterpret_cast<const float2*>(base + L_.td);
  v4.tf32 = s.tf32;
  v4.tw = w.tw;
  v4.twp = L_.twp;
  v4.logrho32 = s.logrho32;
  v4.part = s.part;
  v4.w_out = nullptr;
  v4.ctrl = c->ctrl;

  SplitArgs& x5 = c->sa5;
  const SplitPlan& q5 = c->sp;
  x5.y = s.y;
  x5.shift = shift;
  x5.N = d->N; x5.Kp1 = Kp1; x5.M = M; x5.L = d->L; x5.Lw = Lw;
  x5.nwarps = q5.nwarps; x5.slot_bytes = q5.slot_bytes;
  x5.off_ring = q5.off_ring; x5.off_x = q5.off_x; x5.off_tf = q5.off_tf;
  x5.NP = q5.NP; x5.ncols = q5.ncols;
  x5.k2_off_b = q5.k2_off_b; x5.k2_off_ah = q5.k2_off_ah; x5.k2_off_al = q5.k2_off_al; x5.k2_off_lr = q5.k2_off_lr;
  x5.k2_off_tf = q5.k2_off_tf; x5.k2_off_wt = q5.k2_off_wt; x5.k2_off_ll = q5.k2_off_ll;
  x5.k2_off_cs = q5.k2_off_cs; x5.k2_off_td = q5.k2_off_td; x5.k2_off_info = q5.k2_off_info;
  x5.k2_ndp = q5.k2_ndp;
  x5.wrap = !dense && Lw == d->L ? 1 : 0;
  x5.l0m = ((l0 % d->L) + d->L) % d->L;
  x5.nd = x5.wrap ? d->L / 2 + 1 : Lw;
  x5.twp = L_.twp;
  x5.two_beta = s.two_beta;
  x5.x32 = s.x32;
  x5.tf32 = s.tf32;
  x5.td = reinterpret_cast<const float2*>(base + L_.td);
  x5.tw = dense ? s.tw : nullptr;
  x5.logrho32 = s.logrho32;
  x5.tcb = base + L_.tcb;
  x5.cbuf = reinterpret_cast<float2*>(base + L_.cbuf);
  x5.wbuf = reinterpret_cast<float2*>(base + L_.wbuf);
  x5.part = s.part;
  x5.G = G;
  x5.w_out = nullptr;
  x5.ctrl = c->ctrl;

  SetupArgs& u = c->su;
  u.N = d->N; u.Kp1 = Kp1; u.Q = d->Q; u.M = M; u.L = d->L; u.Lw = Lw;
  u.l0 = l0; u.twp = L_.twp; u.kp4 = L_.kp4; u.sigma2 = d->sigma2;
  u.step = step; u.dense = dense ? 1 : 0;
  u.x_in = nullptr; u.log_rho_in = nullptr; u.log_rho_bar = nullptr; u.gamma_a_inv = nullptr;
  u.tf32 = reinterpret_cast<float2*>(base + L_.tf32);
  u.tf64 = reinterpret_cast<double2*>(base + L_.tf64);
  u.tw = reinterpret_cast<float2*>(base + L_.tw);
  u.tw64 = reinterpret_cast<double2*>(base + L_.tw64);
  u.x32 = reinterpret_cast<float2*>(base + L_.x32);
  u.x64 = reinterpret_cast<double2*>(base + L_.x64);
  u.inv_den = reinterpret_cast<double*>(base + L_.inv_den);
  u.logrho32 = reinterpret_cast<float*>(base + L_.logrho32);
  u.rho64 = reinterpret_cast<double*>(base + L_.rho64);
  u.rhobar64 = reinterpret_cast<double*>(base + L_.rhobar64);
  u.units = reinterpret_cast<int2*>(base + L_.units);
  u.tu = reinterpret_cast<float2*>(base + L_.tu);
  u.td = reinterpret_cast<float2*>(base + L_.td);
  u.nd = c->vs ? x5.nd : c->v3 ? c->v3p.nd : c->v4 ? c->v4p.nd : c->v2 ? v.nd : 0;
  u.nu = nu;
  u.nup = nup;
  u.ctrl = c->ctrl;

  UpdateArgs& up = c->ua;
  up.N = d->N; up.Kp1 = Kp1; up.Q = d->Q; up.M = M; up.L = d->L; up.Lw = Lw;
  up.sigma2 = d->sigma2; up.beta = 1.0 / d->sigma2; up.gamma = 0.0; up.tol = 0.0;
  up.ll_const = (double)d->N * (double)M * std::log(kPi * d->sigma2);
  up.update_rho = 0; up.max_iters = 1 << 30;
  up.tot = c->tot; up.cols = L_.cols;
  up.x64 = u.x64; up.x32 = u.x32; up.inv_den = u.inv_den; up.rho64 = u.rho64; up.logrho32 = u.logrho32;
  up.rhobar64 = u.rhobar64; up.tf64 = u.tf64; up.tf32 = u.tf32; up.ctrl = c->ctrl;
  up.stats = nullptr; up.x_traj = nullptr; up.x_out = nullptr; up.log_rho_out = nullptr;
  up.loglik_out = nullptr; up.step_out = nullptr;
  c->update_smem = update_xf_offset(M, d->L, Kp1) + 16 * M;
  if (c->update_smem > 48 * 1024 && raise_smem_limit(reinterpret_cast<const void*>(k_finalize), c->update_smem) != MRA_OK)
    return MRA_ECUDA;
  c->reduce_blocks = (L_.cols + 7) / 8;
  // about one column per warp, in one wave (the finalize's CTAs hold the update's shared memory)
  c->fin_blocks = std::max(1, std::min(G, (L_.cols + 15) / 16));
  return MRA_OK;
}

int launch_setup(const EmCall& c, cudaStream_t st) {
  const int n = std::max(std::max(c.su.L, c.su.M), c.su.Lw);
  const int blocks = std::min(1024, (n + 127) / 128);
  k_setup<<<blocks, 128, 0, st>>>(c.su);
  if (c.vs) {
    const int ntd = c.su.Kp1 * c.su.nd;
    k_setup_td<<<std::min(1024, (ntd + 255) / 256), 256, 0, st>>>(c.su);
    if (c.su.dense) {
      const int ntw = c.su.kp4 * c.su.twp;
      k_setup_tw<<<std::min(1024, (ntw + 255) / 256), 256, 0, st>>>(c.su);
    }
    const int nb = c.sp.NP * c.sp.KA;
    k_setup_tcb<<<std::min(1024, (nb + 255) / 256), 256, 0, st>>>(
        c.su, reinterpret_cast<__half*>(const_cast<void*>(c.sa5.tcb)), c.sp.NP, c.sp.KA);
  } else if (c.v3 || c.v4) {
    const int ntd = c.su.Kp1 * c.su.nd;
    k_setup_td<<<std::min(1024, (ntd + 255) / 256), 256, 0, st>>>(c.su);
    if (c.su.dense) {  // the rotation to each image's reference
      const int ntw = c.su.kp4 * c.su.twp;
      k_setup_tw<<<std::min(1024, (ntw + 255) / 256), 256, 0, st>>>(c.su);
    }
  } else if (c.v2) {
    k_setup_units<<<1, 32, 0, st>>>(c.su);
    const int ntu = c.su.Kp1 * c.su.nup;
    k_setup_tu<<<std::min(1024, (ntu + 255) / 256), 256, 0, st>>>(c.su);
    const int ntd = c.su.Kp1 * c.su.nd;  // pass 2 around each image's peak
    k_setup_td<<<std::min(1024, (ntd + 255) / 256), 256, 0, st>>>(c.su);
    if (c.su.dense) {  // the rotation to each image's peak
      const int ntw = c.su.kp4 * c.su.twp;
      k_setup_tw<<<std::min(1024, (ntw + 255) / 256), 256, 0, st>>>(c.su);
    }
  } else {
    const int ntw = c.su.kp4 * c.su.twp;
    k_setup_tw<<<std::min(1024, (ntw + 255) / 256), 256, 0, st>>>(c.su);
  }
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

void launch_sweep(const EmCall& c, cudaStream_t st) {
  if (c.vs) {
    c.sp.fns.corr<<<c.lay.G, kTcStreamThreads, c.sp.smem1, st>>>(c.sa5);
    c.sp.trans<<<c.lay.G, kTcTransThreads, c.sp.smem2, st>>>(c.sa5);
    c.sp.fns.accum<<<c.lay.G, kTcStreamThreads, c.sp.smem1, st>>>(c.sa5);
  } else if (c.v4)
    c.v4p.launch.fn<<<c.lay.G, c.v4p.launch.threads, c.v4p.smem, st>>>(c.sa4);
  else if (c.v3)
    c.v3p.fn<<<c.lay.G, kV3Threads, c.v3p.smem, st>>>(c.sa3);
  else if (c.v6)
    c.v6p.launch.fn<<<c.lay.G, c.v6p.launch.threads, c.v6p.smem, st>>>(c.sa6);
  else if (c.v2)
    c.v2p.launch.fn<<<c.lay.G, c.v2p.launch.threads, c.v2p.smem, st>>>(c.sa2);
  else
    c.sweep<<<c.lay.G, kSweepThreads, c.plan.smem, st>>>(c.sa);
}

int launch_iteration(const EmCall& c, cudaStream_t st, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr) {
  // external event nodes: inside stream capture a plain record would only add a dependency edge
  if (ev0 && cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal) != cudaSuccess) return MRA_ECUDA;
  launch_sweep(c, st);
  if (ev1 && cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal) != cudaSuccess) return MRA_ECUDA;
  k_finalize<<<c.fin_blocks, kUpdateThreads, c.update_smem, st>>>(c.ua, c.sa.part, c.lay.G, c.lay.cols);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

// The window's rotation spacing: step (0 is read as 1, the grid).
double param_step(const mra_em_params* p) { return p->step == 0.0 ? 1.0 : p->step; }

int check_params(const mra_dims* d, const mra_em_params* p) {
  if (!p) return MRA_EINVAL;
  if (!window_ok(d->L, p->Lw, p->l0, param_step(p))) return MRA_EINVAL;
  if (!(p->gamma >= 0.0) || !isfinite(p->gamma)) return MRA_EINVAL;
  if (p->gamma > 0.0 && !ptr_ok(p->log_rho_bar, 8)) return MRA_EINVAL;
  if (p->gamma_a_inv && !ptr_ok(p->gamma_a_inv, 8)) return MRA_EINVAL;
  return MRA_OK;
}

}  // namespace
}  // namespace mra

using namespace mra;

// ---------------------------------------------------------------- entry points (C ABI)
extern "C" {

MRA_API const char* mra_status_string(int s) {
  switch (s) {
    case MRA_OK: return "ok";
    case MRA_EINVAL: return "invalid argument";
    case MRA_ENOMEM: return "host allocation failed";
    case MRA_ECUDA: return "CUDA runtime error";
    case MRA_ETIMEOUT: return "device wait timed out";
    case MRA_ENUMERIC: return "non-finite value";
    case MRA_EWORKSPACE: return "workspace too small";
    default: return "unknown status";
  }
}

MRA_API int mra_device_info(int32_t* num_sms, int32_t* sweep_grid_out) {
  DevInfo d;
  const int st = dev_info(&d);
  if (st != MRA_OK) return st;
  if (num_sms) *num_sms = d.sms;
  if (sweep_grid_out) *sweep_grid_out = d.sms;
  return MRA_OK;
}

MRA_API size_t mra_em_workspace_bytes(const mra_dims* d, int32_t Lw) {
  if (check_dims(d) != MRA_OK || Lw < 1) return 0;
  DevInfo di;
  if (dev_info(&di) != MRA_OK) return 0;
  return em_layout(d->N, d->K, d->Q, d->L, Lw, di.sms * kMaxCtasPerSm).total;
}

}  // extern "C"

static int em_step_impl(const mra_dims* d, const mra_em_params* p, const float* y, int yfmt, const int32_t* shift,
                        const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                        double* loglik_out, double* step_out, float* w_out, void* ws, size_t ws_bytes,
                        void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if ((st = check_params(d, p)) != MRA_OK) return st;
  if (!ptr_ok(x_in, 16) || !ptr_ok(log_rho_in, 8) || !ptr_ok(x_out, 16) || !ptr_ok(log_rho_out, 8))
    return MRA_EINVAL;
  if (w_out && !ptr_ok(w_out, 4)) return MRA_EINVAL;
  EmCall c;
  if ((st = prepare(d, p->Lw, p->l0, param_step(p), y, shift, ws, ws_bytes, &c, true, yfmt)) != MRA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c.su.x_in = reinterpret_cast<const double2*>(x_in);
  c.su.log_rho_in = log_rho_in;
  c.su.log_rho_bar = p->gamma > 0.0 ? p->log_rho_bar : nullptr;
  c.su.gamma_a_inv = p->gamma_a_inv;
  c.set_w_out(w_out);
  c.ua.gamma = p->gamma;
  c.ua.update_rho = p->update_rho ? 1 : 0;
  c.ua.x_out = reinterpret_cast<double2*>(x_out);
  c.ua.log_rho_out = log_rho_out;
  c.ua.loglik_out = loglik_out;
  c.ua.step_out = step_out;
  if ((st = launch_setup(c, s)) != MRA_OK) return st;
  return launch_iteration(c, s);
}

static int em_run_impl(const mra_dims* d, const mra_em_params* p, const float* y, int yfmt, const int32_t* shift,
                       double* x_inout, double* log_rho_inout, int32_t* iters_out, double* stats_out,
                       double* x_traj_out, void* ws, size_t ws_bytes, void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if ((st = check_params(d, p)) != MRA_OK) return st;
  if (p->max_iters < 1 || p->check_every < 1) return MRA_EINVAL;
  if (!ptr_ok(x_inout, 16) || !ptr_ok(log_rho_inout, 8)) return MRA_EINVAL;
  if (stats_out && !ptr_ok(stats_out, 8)) return MRA_EINVAL;
  if (x_traj_out && !ptr_ok(x_traj_out, 16)) return MRA_EINVAL;
  EmCall c;
  if ((st = prepare(d, p->Lw, p->l0, param_step(p), y, shift, ws, ws_bytes, &c, true, yfmt)) != MRA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c.su.x_in = reinterpret_cast<const double2*>(x_inout);
  c.su.log_rho_in = log_rho_inout;
  c.su.log_rho_bar = p->gamma > 0.0 ? p->log_rho_bar : nullptr;
  c.su.gamma_a_inv = p->gamma_a_inv;
  c.ua.gamma = p->gamma;
  c.ua.tol = p->tol;
  c.ua.update_rho = p->update_rho ? 1 : 0;
  c.ua.max_iters = p->max_iters;
  c.ua.stats = stats_out;
  c.ua.x_traj = reinterpret_cast<double2*>(x_traj_out);
  if ((st = launch_setup(c, s)) != MRA_OK) return st;

  const int chunk = std::min(p->check_every, p->max_iters);
  const bool timed = p->sweep_ms != nullptr;
  std::vector<cudaEvent_t> ev;
  int rc = MRA_OK;
  if (timed) {
    ev.assign(2 * chunk, nullptr);
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) rc = MRA_ECUDA;
  }
  cudaStream_t cap = nullptr;
  if (rc == MRA_OK && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) rc = MRA_ECUDA;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (rc == MRA_OK && cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MRA_ECUDA;
  if (rc == MRA_OK) {
    for (int i = 0; i < chunk && rc == MRA_OK; ++i)
      rc = launch_iteration(c, cap, timed ? ev[2 * i] : nullptr, timed ? ev[2 * i + 1] : nullptr);
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess) rc = MRA_ECUDA;
  }
  if (rc == MRA_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = MRA_ECUDA;
  Ctrl host_ctrl{};
  const int launches = (p->max_iters + chunk - 1) / chunk;
  for (int i = 0; i < launches && rc == MRA_OK; ++i) {
    if (cudaGraphLaunch(exec, s) != cudaSuccess) { rc = MRA_ECUDA; break; }
    if ((p->tol > 0.0 && i + 1 < launches) || timed) {
      const int before = host_ctrl.iter;
      if (cudaMemcpyAsync(&host_ctrl, c.ctrl, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = MRA_ECUDA;
        break;
      }
      if (timed) {
        for (int j = 0; j < chunk && before + j < host_ctrl.iter; ++j) {
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, ev[2 * j], ev[2 * j + 1]) != cudaSuccess) { rc = MRA_ECUDA; break; }
          p->sweep_ms[before + j] = ms;
        }
      }
      if (host_ctrl.done || host_ctrl.status != MRA_OK) break;
    }
  }
  if (rc == MRA_OK) {
    k_export<<<std::max(1, (std::max(c.lay.M, p->Lw) + 255) / 256), 256, 0, s>>>(
        c.lay.M, p->Lw, c.su.x64, c.su.rho64, reinterpret_cast<double2*>(x_inout), log_rho_inout);
    if (cudaGetLastError() != cudaSuccess) rc = MRA_ECUDA;
  }
  if (rc == MRA_OK) {
    if (cudaMemcpyAsync(&host_ctrl, c.ctrl, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = MRA_ECUDA;
    else {
      if (iters_out) *iters_out = host_ctrl.iter;
      if (host_ctrl.status != MRA_OK) rc = host_ctrl.status;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  for (auto e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

extern "C" {

MRA_API int mra_em_step(const mra_dims* d, const mra_em_params* p, const float* y, const int32_t* shift,
                        const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                        double* loglik_out, double* step_out, float* w_out, void* ws, size_t ws_bytes,
                        void* stream) {
  return em_step_impl(d, p, y, 0, shift, x_in, log_rho_in, x_out, log_rho_out, loglik_out, step_out, w_out, ws,
                      ws_bytes, stream);
}

MRA_API int mra_em_step_hl(const mra_dims* d, const mra_em_params* p, const void* y_hl, const int32_t* shift,
                           const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                           double* loglik_out, double* step_out, float* w_out, void* ws, size_t ws_bytes,
                           void* stream) {
  return em_step_impl(d, p, static_cast<const float*>(y_hl), 1, shift, x_in, log_rho_in, x_out, log_rho_out,
                      loglik_out, step_out, w_out, ws, ws_bytes, stream);
}

MRA_API int mra_em_run(const mra_dims* d, const mra_em_params* p, const float* y, const int32_t* shift,
                       double* x_inout, double* log_rho_inout, int32_t* iters_out, double* stats_out,
                       double* x_traj_out, void* ws, size_t ws_bytes, void* stream) {
  return em_run_impl(d, p, y, 0, shift, x_inout, log_rho_inout, iters_out, stats_out, x_traj_out, ws, ws_bytes,
                     stream);
}

MRA_API int mra_em_run_hl(const mra_dims* d, const mra_em_params* p, const void* y_hl, const int32_t* shift,
                          double* x_inout, double* log_rho_inout, int32_t* iters_out, double* stats_out,
                          double* x_traj_out, void* ws, size_t ws_bytes, void* stream) {
  return em_run_impl(d, p, static_cast<const float*>(y_hl), 1, shift, x_inout, log_rho_inout, iters_out, stats_out,
                     x_traj_out, ws, ws_bytes, stream);
}

// y (complex64) -> BF16 hi/lo split: per pair of complex values, bf16 hi of (re, im, re, im)
// then bf16 lo of the residuals, both rounded to nearest even.
__global__ void k_split_bf16(const float4* y, long long groups, uint4* out) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
    const float4 v = y[g];
    const float f[4] = {v.x, v.y, v.z, v.w};
    unsigned short h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const __nv_bfloat16 bh = __float2bfloat16_rn(f[t]);
      const __nv_bfloat16 bl = __float2bfloat16_rn(f[t] - __bfloat162float(bh));
      h[t] = __bfloat16_as_ushort(bh);
      l[t] = __bfloat16_as_ushort(bl);
    }
    out[g] = make_uint4(h[0] | ((unsigned)h[1] << 16), h[2] | ((unsigned)h[3] << 16), l[0] | ((unsigned)l[1] << 16),
                        l[2] | ((unsigned)l[3] << 16));
  }
}

MRA_API int mra_y_split_bf16(const float* y, int64_t count, void* y_hl_out, void* stream) {
  if (count < 0 || count % 2 != 0) return MRA_EINVAL;
  if (count == 0) return MRA_OK;
  if (!ptr_ok(y, 16) || !ptr_ok(y_hl_out, 16)) return MRA_EINVAL;
  const long long groups = count / 2;
  const int blocks = (int)std::min<long long>((groups + 255) / 256, 152LL * 16);
  k_split_bf16<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(reinterpret_cast<const float4*>(y), groups,
                                                                        static_cast<uint4*>(y_hl_out));
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

// ---------------------------------------------------------------- autotuner and batched runs

}  // extern "C"

namespace mra {
namespace {

constexpr int kBatchedImagesPerCta = 64;

// Sweep candidates the autotuner times, in the order of the default preference (a later candidate
// replaces the best so far only when it is at least 1% faster, so near-ties keep the earlier one).
const SweepSel kTuneCandidates[] = {{4, 0, 0},  {6, 0, 0},  {5, 0, 0},  {1, 0, 0},  {2, 16, 2}, {2, 12, 2}, {2, 8, 3},  {2, 8, 2}, {2, 4, 3},
                                    {2, 4, 2},  {3, 64, 2}, {3, 32, 2}, {3, 16, 2}, {3, 128, 1},
                                    {3, 64, 1}, {3, 32, 1}};

// Best of `reps` timed sweeps (after one untimed) of a prepared call whose setup has run; < 0 on error.
float time_sweep(const EmCall& c, cudaStream_t s, int reps) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = -1.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    launch_sweep(c, s);
    for (int r = 0; r < reps; ++r) {
      float ms = 0.f;
      if (cudaEventRecord(e0, s) != cudaSuccess) break;
      launch_sweep(c, s);
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        break;
      if (best < 0.f || ms < best) best = ms;
    }
  }
  if (cudaGetLastError() != cudaSuccess) best = -1.f;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return best;
}

int autotune_impl(const mra_dims* d, const mra_em_params* p, const float* y, int yfmt, const int32_t* shift,
                  const double* x, const double* log_rho, void* ws, size_t ws_bytes, cudaStream_t s, SweepSel* out) {
  SweepSel best{0, 0, 0};
  float best_ms = -1.f;
  for (const SweepSel& cand : kTuneCandidates) {
    EmCall c;
    const int st = prepare(d, p->Lw, p->l0, param_step(p), y, shift, ws, ws_bytes, &c, true, yfmt, &cand);
    if (st == MRA_EINVAL) continue;  // this candidate cannot take the shape
    if (st != MRA_OK) return st;
    if (cand.kind == 2 && ((cand.bi && c.v3p.bi != cand.bi) || (cand.ns && c.v3p.ns != cand.ns))) continue;
    if (cand.kind == 3 && ((cand.bi && (1 << c.v4p.lc) != cand.bi) ||
                           (cand.ns && c.v4p.launch.ctas_per_sm != cand.ns)))
      continue;
    c.su.x_in = reinterpret_cast<const double2*>(x);
    c.su.log_rho_in = log_rho;
    int rc = launch_setup(c, s);
    if (rc != MRA_OK) return rc;
    const float ms = time_sweep(c, s, 2);
    if (ms < 0.f) return MRA_ECUDA;
    if (best_ms < 0.f || ms < 0.99f * best_ms) best_ms = ms, best = cand;
  }
  if (best_ms >= 0.f) tune_store(tune_key(d, p->Lw, p->l0, param_step(p), yfmt), best);
  if (out) *out = best;
  return MRA_OK;
}

// Bytes after the instances' workspaces in a batched workspace: the persistent kernel's instance
// table, its item counters and its grid barrier.
size_t batched_extra_bytes(int n, int tmax) {
  return align256(sizeof(BatchedInst) * (size_t)n) + align256(sizeof(unsigned) * (2 * (size_t)tmax + 2));
}
constexpr int kNotPersistent = 1;  // run_batched_persistent: some instance has no persistent body
constexpr size_t kBatchedTileBytes = (size_t)1 << 20;  // default y bytes per persistent sweep item

// Instantiated graphs of batched runs, keyed by the exact instance list, workspace and
// device: a repeated call with the same list launches the same graph again.
struct BatchedGraph {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec;
  std::vector<Ctrl*> ctrl;
};
std::mutex g_graph_mu;
std::map<std::vector<unsigned char>, size_t> g_tiles;  // persistent batched runs: the tuned tile
std::vector<BatchedGraph> g_graphs;  // most recent last
constexpr size_t kGraphCache = 4;

std::vector<unsigned char> batched_key(const mra_instance* inst, int n, const void* ws, size_t ws_bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<unsigned char> k(sizeof(mra_instance) * n + sizeof(ws) + sizeof(ws_bytes) + sizeof(dev));
  unsigned char* o = k.data();
  memcpy(o, inst, sizeof(mra_instance) * n);
  o += sizeof(mra_instance) * n;
  memcpy(o, &ws, sizeof(ws));
  o += sizeof(ws);
  memcpy(o, &ws_bytes, sizeof(ws_bytes));
  o += sizeof(ws_bytes);
  memcpy(o, &dev, sizeof(dev));
  return k;
}

// The persistent path of mra_em_run_batched: every instance runs the lean warp sweep (or, for windows
// it cannot take, the warp sweep's any-window instance) as items of one cooperative kernel.
// Returns kNotPersistent if some instance has no body in that kernel.
int run_batched_persistent(const mra_instance* inst, int n, int tune, int32_t* iters_out, float* exec_ms_out,
                           unsigned char* base, const std::vector<size_t>& off, cudaStream_t s,
                           std::vector<unsigned char> key) {
  key.push_back(1);  // the persistent kernel's graph and tile, not the per-instance graph
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != MRA_OK) return rc;
  const int cap = di.max_smem_optin - batched_static_smem() - 256;
  int tmax = 0;
  for (int i = 0; i < n; ++i) {
    if (inst[i].y_format != 0) return kNotPersistent;
    tmax = std::max(tmax, inst[i].prm.max_iters);
  }
  std::vector<EmCall> calls(n);
  std::vector<BatchedInst> hb(n);
  std::vector<int> gmax(n);
  int smem = 0;
  for (int i = 0; i < n; ++i) {
    const mra_instance& a = inst[i];
    EmCall& c = calls[i];
    const SweepSel lean{4, 0, 0}, warp{1, 0, 0};
    const float* y = static_cast<const float*>(a.y);
    rc = prepare(&a.dims, a.prm.Lw, a.prm.l0, param_step(&a.prm), y, a.shift, base + off[i], off[i + 1] - off[i], &c,
                 true, 0, &lean, cap);
    if (rc == MRA_EINVAL)
      rc = prepare(&a.dims, a.prm.Lw, a.prm.l0, param_step(&a.prm), y, a.shift, base + off[i], off[i + 1] - off[i],
                   &c, true, 0, &warp, cap);
    if (rc == MRA_EINVAL) return kNotPersistent;
    if (rc != MRA_OK) return rc;
    const int body = batched_body_id(a.dims.Q, c.v5, (a.dims.K + 1 + 7) / 8, c.sa2.NUP, c.v2p.lwc);
    if (body < 0) return kNotPersistent;
    gmax[i] = c.lay.G;
    c.su.x_in = reinterpret_cast<const double2*>(a.x_inout);
    c.su.log_rho_in = a.log_rho_inout;
    c.su.log_rho_bar = a.prm.gamma > 0.0 ? a.prm.log_rho_bar : nullptr;
    c.su.gamma_a_inv = a.prm.gamma_a_inv;
    c.ua.gamma = a.prm.gamma;
    c.ua.tol = a.prm.tol;
    c.ua.update_rho = a.prm.update_rho ? 1 : 0;
    c.ua.max_iters = a.prm.max_iters;
    c.ua.stats = a.stats_out;
    BatchedInst& bi = hb[i];
    bi.ua = c.ua;
    bi.body = body;
    bi.cols = c.lay.cols;
    bi.part = c.sa.part;
    bi.tot = c.tot;
    bi.ctrl = c.ctrl;
    smem = std::max(smem, std::max(c.v2p.smem, c.update_smem));
  }
  BatchedInst* dinst = reinterpret_cast<BatchedInst*>(base + off[n]);
  unsigned* counters = reinterpret_cast<unsigned*>(base + off[n] + align256(sizeof(BatchedInst) * (size_t)n));
  const size_t cnt_bytes = sizeof(unsigned) * (2 * (size_t)tmax + 2);
  // Tile: about `tile_bytes` of y per sweep item, so that items of instances with long and short rows
  // take similar times and the CTAs reach each grid barrier together.
  int items = 0;
  auto assign = [&](size_t tile_bytes) -> int {
    items = 0;
    for (int i = 0; i < n; ++i) {
      const size_t img = (size_t)calls[i].lay.M * 8;
      const size_t want = ((size_t)inst[i].dims.N * img + tile_bytes - 1) / tile_bytes;
      const int slots = (int)std::max<size_t>(1, std::min<size_t>((size_t)gmax[i], want));
      calls[i].lay.G = slots;
      calls[i].sa2.G = slots;
      hb[i].sa = calls[i].sa2;
      hb[i].slots = slots;
      hb[i].first_item = items;
      items += slots;
    }
    if (cudaMemcpyAsync(dinst, hb.data(), sizeof(BatchedInst) * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return MRA_ECUDA;
    return MRA_OK;
  };
  size_t tile_bytes = kBatchedTileBytes;
  if (const char* e = getenv("MRA_BATCHED_TILE_KB")) tile_bytes = (size_t)std::max(16, atoi(e)) * 1024;
  bool have_tile = false;
  {
    std::lock_guard<std::mutex> g(g_graph_mu);
    auto it = g_tiles.find(key);
    if (it != g_tiles.end()) tile_bytes = it->second, have_tile = true;
  }
  BatchedArgs ba;
  ba.inst = dinst;
  ba.n = n;
  ba.items = items;
  ba.iters = tmax;
  ba.counters = counters;
  ba.barrier = counters + 2 * tmax;
  ba.status = &calls[0].ctrl->status;  // a grid barrier that gives up reports through the first instance
  ba.limit_ns = kWaitLimitNs;
  // the run: counters cleared, setups, the persistent kernel (all iterations, or one for tuning), exports
  auto record = [&](cudaStream_t st, bool tuning = false) -> int {
    if (cudaMemsetAsync(counters, 0, cnt_bytes, st) != cudaSuccess) return MRA_ECUDA;
    for (int i = 0; i < n; ++i) {
      const int r = launch_setup(calls[i], st);
      if (r != MRA_OK) return r;
    }
    BatchedArgs b2 = ba;
    b2.items = items;
    if (tuning) b2.iters = 1;
    const int r = launch_em_batched(b2, di.sms, smem, st);
    if (r != MRA_OK) return r;
    if (tuning) return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
    for (int i = 0; i < n; ++i) {
      const int Lw = inst[i].prm.Lw, M = calls[i].lay.M;
      k_export<<<std::max(1, (std::max(M, Lw) + 255) / 256), 256, 0, st>>>(
          M, Lw, calls[i].su.x64, calls[i].su.rho64, reinterpret_cast<double2*>(inst[i].x_inout), inst[i].log_rho_inout);
    }
    return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
  };
  std::vector<Ctrl*> ctrl(n);
  for (int i = 0; i < n; ++i) ctrl[i] = calls[i].ctrl;
  auto finish = [&](cudaEvent_t t0, cudaEvent_t t1) -> int {
    int r = MRA_OK;
    if (cudaEventSynchronize(t1) != cudaSuccess) r = MRA_ECUDA;
    if (r == MRA_OK && exec_ms_out && cudaEventElapsedTime(exec_ms_out, t0, t1) != cudaSuccess) r = MRA_ECUDA;
    for (int i = 0; i < n && r == MRA_OK; ++i) {
      Ctrl h{};
      if (cudaMemcpy(&h, ctrl[i], 16, cudaMemcpyDeviceToHost) != cudaSuccess) {
        r = MRA_ECUDA;
        break;
      }
      if (iters_out) iters_out[i] = h.iter;
      if (h.status != MRA_OK) r = h.status;
    }
    return r;
  };
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) rc = MRA_ECUDA;
  // the autotuner's part: one iteration of the persistent kernel per tile candidate (no export, so the
  // instances' x and log rho are not touched), the fastest kept for this instance list
  if (rc == MRA_OK && tune && !have_tile && !getenv("MRA_BATCHED_TILE_KB")) {
    float best = -1.f;
    for (const size_t cand : {(size_t)512 << 10, (size_t)1 << 20, (size_t)2 << 20, (size_t)4 << 20}) {
      if ((rc = assign(cand)) != MRA_OK) break;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == MRA_OK; ++rep) {
        if (cudaEventRecord(t0, s) != cudaSuccess) rc = MRA_ECUDA;
        if (rc == MRA_OK) rc = record(s, true);
        if (rc == MRA_OK && (cudaEventRecord(t1, s) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess))
          rc = MRA_ECUDA;
      }
      if (rc == MRA_OK && (best < 0.f || ms < best)) best = ms, tile_bytes = cand;
    }
    for (int i = 0; i < n && rc == MRA_OK; ++i) {  // a timed-out tuning run must not pass silently
      Ctrl h{};
      if (cudaMemcpy(&h, calls[i].ctrl, 16, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MRA_ECUDA;
      else if (h.status != MRA_OK) rc = h.status;
    }
    if (rc == MRA_OK) {
      std::lock_guard<std::mutex> g(g_graph_mu);
      g_tiles[key] = tile_bytes;
    }
  }
  if (rc == MRA_OK) rc = assign(tile_bytes);
  cudaGraphExec_t cached = nullptr;
  {
    std::lock_guard<std::mutex> g(g_graph_mu);
    for (auto& e : g_graphs)
      if (e.key == key) cached = e.exec;
  }
  if (rc == MRA_OK && !cached) {  // capture the run as a graph (or, if capture fails, launch it directly)
    cudaStream_t capst = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool captured = false;
    if (cudaStreamCreateWithFlags(&capst, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamBeginCapture(capst, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int r = record(capst);
      const bool ended = cudaStreamEndCapture(capst, &graph) == cudaSuccess;
      captured = r == MRA_OK && ended && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    }
    cudaGetLastError();  // a failed capture leaves an error behind; the direct launch below decides
    if (graph) cudaGraphDestroy(graph);
    if (capst) cudaStreamDestroy(capst);
    if (captured) {
      std::lock_guard<std::mutex> g(g_graph_mu);
      if (g_graphs.size() >= kGraphCache) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
      }
      g_graphs.push_back(BatchedGraph{key, exec, ctrl});
      cached = exec;
    } else {
      if (exec) cudaGraphExecDestroy(exec);
      if (cudaEventRecord(t0, s) != cudaSuccess) rc = MRA_ECUDA;
      if (rc == MRA_OK) rc = record(s);
      if (rc == MRA_OK && cudaEventRecord(t1, s) != cudaSuccess) rc = MRA_ECUDA;
      if (rc == MRA_OK) rc = finish(t0, t1);
    }
  }
  if (rc == MRA_OK && cached) {
    if (cudaEventRecord(t0, s) != cudaSuccess || cudaGraphLaunch(cached, s) != cudaSuccess ||
        cudaEventRecord(t1, s) != cudaSuccess)
      rc = MRA_ECUDA;
    if (rc == MRA_OK) rc = finish(t0, t1);
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  return rc;
}

}  // namespace
}  // namespace mra

extern "C" {

MRA_API int mra_em_autotune(const mra_dims* d, const mra_em_params* p, const void* y, int32_t y_format,
                            const int32_t* shift, const double* x, const double* log_rho, int32_t* choice_out,
                            void* ws, size_t ws_bytes, void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if ((st = check_params(d, p)) != MRA_OK) return st;
  if ((y_format != 0 && y_format != 1) || !ptr_ok(x, 16) || !ptr_ok(log_rho, 8)) return MRA_EINVAL;
  SweepSel sel{0, 0, 0};
  st = autotune_impl(d, p, static_cast<const float*>(y), y_format, shift, x, log_rho, ws, ws_bytes,
                     static_cast<cudaStream_t>(stream), &sel);
  if (st == MRA_OK && choice_out) {
    choice_out[0] = sel.kind;
    choice_out[1] = sel.bi;
    choice_out[2] = sel.ns;
  }
  return st;
}

MRA_API size_t mra_em_batched_workspace_bytes(const mra_instance* inst, int32_t n) {
  if (!inst || n < 1) return 0;
  size_t total = 0;
  int tmax = 0;
  for (int i = 0; i < n; ++i) {
    total += align256(mra_em_workspace_bytes(&inst[i].dims, std::max(inst[i].prm.Lw, 1)));
    tmax = std::max(tmax, inst[i].prm.max_iters);
  }
  return total + batched_extra_bytes(n, tmax);
}

MRA_API int mra_em_run_batched(const mra_instance* inst, int32_t n, int32_t tune, int32_t* iters_out,
                               float* exec_ms_out, void* ws, size_t ws_bytes, void* stream) {
  if (!inst || n < 1 || !ptr_ok(ws, 256)) return MRA_EINVAL;
  if (ws_bytes < mra_em_batched_workspace_bytes(inst, n)) return MRA_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const mra_instance& a = inst[i];
    int st = check_dims(&a.dims);
    if (st == MRA_OK) st = check_params(&a.dims, &a.prm);
    if (st != MRA_OK) return st;
    if (a.prm.max_iters < 1 || (a.y_format != 0 && a.y_format != 1)) return MRA_EINVAL;
    if (!ptr_ok(a.x_inout, 16) || !ptr_ok(a.log_rho_inout, 8)) return MRA_EINVAL;
    if (a.stats_out && !ptr_ok(a.stats_out, 8)) return MRA_EINVAL;
    off[i + 1] = off[i] + align256(mra_em_workspace_bytes(&a.dims, a.prm.Lw));
  }
  unsigned char* base = static_cast<unsigned char*>(ws);
  const std::vector<unsigned char> key = batched_key(inst, n, ws, ws_bytes);
  auto run_cached = [&](cudaGraphExec_t exec, const std::vector<Ctrl*>& ctrl) -> int {
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    int rc = MRA_OK;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) rc = MRA_ECUDA;
    if (rc == MRA_OK && (cudaEventRecord(t0, s) != cudaSuccess || cudaGraphLaunch(exec, s) != cudaSuccess ||
                         cudaEventRecord(t1, s) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess))
      rc = MRA_ECUDA;
    if (rc == MRA_OK && exec_ms_out && cudaEventElapsedTime(exec_ms_out, t0, t1) != cudaSuccess) rc = MRA_ECUDA;
    for (int i = 0; i < n && rc == MRA_OK; ++i) {
      Ctrl h{};
      if (cudaMemcpy(&h, ctrl[i], 16, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = MRA_ECUDA;
        break;
      }
      if (iters_out) iters_out[i] = h.iter;
      if (h.status != MRA_OK) rc = h.status;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return rc;
  };
  if (!tune) {
    std::lock_guard<std::mutex> g(g_graph_mu);
    for (auto& e : g_graphs)
      if (e.key == key) return run_cached(e.exec, e.ctrl);
  }
  // the autotuner runs once per shape not yet in its cache, on the first instance of that shape
  if (tune) {
    for (int i = 0; i < n; ++i) {
      const mra_instance& a = inst[i];
      SweepSel have;
      if (tune_lookup(tune_key(&a.dims, a.prm.Lw, a.prm.l0, param_step(&a.prm), a.y_format), &have)) continue;
      const int st = autotune_impl(&a.dims, &a.prm, static_cast<const float*>(a.y), a.y_format, a.shift, a.x_inout,
                                   a.log_rho_inout, base + off[i], off[i + 1] - off[i], s, nullptr);
      if (st != MRA_OK) return st;
    }
  }
  // one persistent kernel for all instances where every instance has a sweep body in it (the
  // default); MRA_BATCHED=graph keeps the graph of per-instance launches below
  {
    const char* bm = getenv("MRA_BATCHED");
    if (!(bm && strcmp(bm, "graph") == 0)) {
      const int rc = run_batched_persistent(inst, n, tune, iters_out, exec_ms_out, base, off, s, key);
      if (rc != kNotPersistent) return rc;
    }
  }
  std::vector<EmCall> calls(n);
  for (int i = 0; i < n; ++i) {
    const mra_instance& a = inst[i];
    EmCall& c = calls[i];
    const int st = prepare(&a.dims, a.prm.Lw, a.prm.l0, param_step(&a.prm), static_cast<const float*>(a.y), a.shift, base + off[i],
                           off[i + 1] - off[i], &c, true, a.y_format);
    if (st != MRA_OK) return st;
    // a small instance takes few SMs (about one persistent CTA per kBatchedImagesPerCta images),
    // so that the sweeps of several instances run side by side
    if (c.v2 || c.v3 || c.v4) {
      const int cap = std::max(1, (a.dims.N + kBatchedImagesPerCta - 1) / kBatchedImagesPerCta);
      if (cap < c.lay.G) c.lay.G = cap;
      c.sa2.G = c.lay.G;  // the warp sweeps' partial-sum stride is their launch grid
      c.sa6.G = c.lay.G;
    }
    c.su.x_in = reinterpret_cast<const double2*>(a.x_inout);
    c.su.log_rho_in = a.log_rho_inout;
    c.su.log_rho_bar = a.prm.gamma > 0.0 ? a.prm.log_rho_bar : nullptr;
    c.su.gamma_a_inv = a.prm.gamma_a_inv;
    c.ua.gamma = a.prm.gamma;
    c.ua.tol = a.prm.tol;
    c.ua.update_rho = a.prm.update_rho ? 1 : 0;
    c.ua.max_iters = a.prm.max_iters;
    c.ua.stats = a.stats_out;
  }
  // one graph: the instances are independent branches, forked over a few capture streams
  const int S = std::min(n, 32);  // capture streams: concurrent instance chains
  std::vector<cudaStream_t> side(S, nullptr);
  std::vector<cudaEvent_t> join(S, nullptr);
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = MRA_OK;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
    rc = MRA_ECUDA;
  for (int j = 0; j < S && rc == MRA_OK; ++j)
    if (cudaStreamCreateWithFlags(&side[j], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&join[j], cudaEventDisableTiming) != cudaSuccess)
      rc = MRA_ECUDA;
  if (rc == MRA_OK && cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MRA_ECUDA;
  if (rc == MRA_OK) {
    if (cudaEventRecord(fork, cap) != cudaSuccess) rc = MRA_ECUDA;
    for (int j = 0; j < S && rc == MRA_OK; ++j)
      if (cudaStreamWaitEvent(side[j], fork, 0) != cudaSuccess) rc = MRA_ECUDA;
    for (int i = 0; i < n && rc == MRA_OK; ++i) {
      const EmCall& c = calls[i];
      cudaStream_t st = side[i % S];
      rc = launch_setup(c, st);
      for (int t = 0; t < inst[i].prm.max_iters && rc == MRA_OK; ++t) rc = launch_iteration(c, st);
      if (rc == MRA_OK) {
        const int Lw = inst[i].prm.Lw;
        k_export<<<std::max(1, (std::max(c.lay.M, Lw) + 255) / 256), 256, 0, st>>>(
            c.lay.M, Lw, c.su.x64, c.su.rho64, reinterpret_cast<double2*>(inst[i].x_inout), inst[i].log_rho_inout);
        if (cudaGetLastError() != cudaSuccess) rc = MRA_ECUDA;
      }
    }
    for (int j = 0; j < S; ++j) {
      if (cudaEventRecord(join[j], side[j]) != cudaSuccess || cudaStreamWaitEvent(cap, join[j], 0) != cudaSuccess)
        rc = MRA_ECUDA;
    }
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess) rc = MRA_ECUDA;
  }
  if (rc == MRA_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = MRA_ECUDA;
  std::vector<Ctrl*> ctrl(n);
  for (int i = 0; i < n; ++i) ctrl[i] = calls[i].ctrl;
  if (rc == MRA_OK) rc = run_cached(exec, ctrl);
  if (rc == MRA_OK) {  // keep the graph for the next call with the same list
    std::lock_guard<std::mutex> g(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it)
      if (it->key == key) {
        cudaGraphExecDestroy(it->exec);
        g_graphs.erase(it);
        break;
      }
    if (g_graphs.size() >= kGraphCache) {
      cudaGraphExecDestroy(g_graphs.front().exec);
      g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(BatchedGraph{key, exec, ctrl});
    exec = nullptr;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (int j = 0; j < S; ++j) {
    if (side[j]) cudaStreamDestroy(side[j]);
    if (join[j]) cudaEventDestroy(join[j]);
  }
  if (cap) cudaStreamDestroy(cap);
  if (fork) cudaEventDestroy(fork);
  return rc;
}

MRA_API int mra_loglik_grad(const mra_dims* d, int32_t Lw, int32_t l0, double step, const float* y,
                            const int32_t* shift, const double* x, const double* logits, double kappa,
                            double* loglik_out, double* dx_out, double* dlogits_out, double* dkappa_out, void* ws,
                            size_t ws_bytes, void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if (step == 0.0) step = 1.0;
  if (!ptr_ok(x, 16) || !ptr_ok(logits, 8) || !isfinite(kappa)) return MRA_EINVAL;
  if (dx_out && !ptr_ok(dx_out, 16)) return MRA_EINVAL;
  EmCall c;
  if ((st = prepare(d, Lw, l0, step, y, shift, ws, ws_bytes, &c)) != MRA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c.su.x_in = reinterpret_cast<const double2*>(x);
  if ((st = launch_setup(c, s)) != MRA_OK) return st;
  k_setup_vm<<<1, 256, 0, s>>>(d->L, Lw, l0, step, kappa, logits, c.su.rho64, c.su.logrho32);
  launch_sweep(c, s);
  k_reduce_cols<<<c.reduce_blocks, 256, 0, s>>>(c.sa.part, c.lay.G, c.lay.cols, c.tot, c.ctrl);
  GradArgs g;
  g.N = d->N; g.M = c.lay.M; g.L = d->L; g.Lw = Lw; g.l0 = l0; g.step = step;
  g.sigma2 = d->sigma2; g.beta = 1.0 / d->sigma2; g.kappa = kappa;
  g.tot = c.tot; g.cols = c.lay.cols;
  g.x64 = c.su.x64; g.rho64 = c.su.rho64;
  g.loglik_out = loglik_out; g.dx_out = reinterpret_cast<double2*>(dx_out);
  g.dlogits_out = dlogits_out; g.dkappa_out = dkappa_out;
  k_grad<<<1, 256, 0, s>>>(g);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

}  // extern "C"

static int align_into_tot(const mra_dims* d, const float* y, const int32_t* shift, void* ws, size_t ws_bytes,
                          cudaStream_t s, EmCall* c) {
  int st = prepare(d, 1, 0, 1.0, y, shift, ws, ws_bytes, c, /*allow_v3=*/false);  // align mode lives in the warp sweep
  if (st != MRA_OK) return st;
  const bool qeven = (d->Q % 2) == 0;
  const int M = c->lay.M, vec = qeven ? 2 : 1;
  const int ncolmax = (M / vec + kSweepThreads - 1) / kSweepThreads;
  void (*fn)(const float2*, const int*, int, int, int, int, const float2*, double*, int) = nullptr;
  if (qeven) {
    fn = ncolmax <= 1 ? k_align_partial<true, 1> : ncolmax <= 2 ? k_align_partial<true, 2>
       : ncolmax <= 4 ? k_align_partial<true, 4> : k_align_partial<true, 8>;
  } else {
    fn = ncolmax <= 1 ? k_align_partial<false, 1> : ncolmax <= 2 ? k_align_partial<false, 2>
       : ncolmax <= 4 ? k_align_partial<false, 4> : k_align_partial<false, 8>;
  }
  // tables only (x_in unused: point the setup at a zero-length state)
  const int n = d->L;
  SetupArgs u = c->su;
  u.M = 0; u.Lw = 0;
  k_setup<<<std::min(1024, (n + 127) / 128), 128, 0, s>>>(u);
  if (c->v2) {  // the sweep with weight 1 at offset 0 accumulates sum_j y_j e^{+i k theta_hat_j}
    k_setup_units<<<1, 32, 0, s>>>(c->su);
    c->sa2.align_only = 1;
    launch_sweep(*c, s);
  } else {
    fn<<<c->lay.G, kSweepThreads, 0, s>>>(reinterpret_cast<const float2*>(y), shift, d->N, M, d->Q, d->L,
                                          c->su.tf32, c->sa.part, c->lay.G);
  }
  k_reduce_cols<<<(2 * M + 7) / 8, 256, 0, s>>>(c->sa.part, c->lay.G, 2 * M, c->tot, nullptr);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

extern "C" {

MRA_API int mra_align_mean(const mra_dims* d, const float* y, const int32_t* shift, double* x_out, void* ws,
                           size_t ws_bytes, void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if (!ptr_ok(x_out, 16)) return MRA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EmCall c;
  if ((st = align_into_tot(d, y, shift, ws, ws_bytes, s, &c)) != MRA_OK) return st;
  k_scale_out<<<(c.lay.M + 255) / 256, 256, 0, s>>>(c.lay.M, c.tot, 1.0 / d->N, reinterpret_cast<double2*>(x_out));
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_prior_hist(const mra_dims* d, const float* y, const int32_t* shift_true, const int32_t* shift_est,
                           const double* x_true, int32_t* hist_inout, int32_t* center_out, void* ws, size_t ws_bytes,
                           void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if (!ptr_ok(shift_true, 4) || !ptr_ok(shift_est, 4) || !ptr_ok(x_true, 16) || !ptr_ok(hist_inout, 4))
    return MRA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EmCall c;
  if ((st = align_into_tot(d, y, shift_est, ws, ws_bytes, s, &c)) != MRA_OK) return st;
  int* center_ws = reinterpret_cast<int*>(c.tot + c.lay.cols + 4);
  const int csm = (d->K + 1) * 16;
  k_center<<<1, 256, csm, s>>>(d->K + 1, d->Q, d->L, c.tot, 1.0 / d->N, reinterpret_cast<const double2*>(x_true),
                               c.su.tf64, center_ws, center_out);
  k_hist<<<std::min(4096, (d->N + 255) / 256), 256, 0, s>>>(d->N, d->L, shift_true, shift_est, center_ws, hist_inout);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- fixed-scratch variant of mra_em_step
// Scratch for mra_em_step_noalloc: one array per device, loaded with the library's module in
// the current context.  Host code must not use the symbol itself as a device address; the
// address comes from cudaGetSymbolAddress on every call (cheap once the module is loaded), so a
// context that was destroyed and created again is never handed a stale address.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static int noalloc_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return MRA_ECUDA;
  *out = p;
  return MRA_OK;
}

extern "C" {

MRA_API int mra_em_step_noalloc(const mra_dims* d, const mra_em_params* p, const float* y, const int32_t* shift,
                                const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                                double* loglik_out, double* step_out, float* w_out, void* stream) {
  int st = check_dims(d);
  if (st != MRA_OK) return st;
  if ((st = check_params(d, p)) != MRA_OK) return st;
  DevInfo di;
  if ((st = dev_info(&di)) != MRA_OK) return st;
  if (em_layout(d->N, d->K, d->Q, d->L, p->Lw, di.sms * kMaxCtasPerSm).total > kNoAllocScratchBytes)
    return MRA_EWORKSPACE;
  void* scratch = nullptr;
  if ((st = noalloc_scratch(&scratch)) != MRA_OK) return st;
  return mra_em_step(d, p, y, shift, x_in, log_rho_in, x_out, log_rho_out, loglik_out, step_out, w_out, scratch,
                     kNoAllocScratchBytes, stream);
}

// The status word of the fixed scratch: the control block sits at its start, as in every
// EM workspace, so the same read-and-clear as mra_ws_status applies.
MRA_API int mra_em_step_noalloc_status(void* stream) {
  void* scratch = nullptr;
  const int st = noalloc_scratch(&scratch);
  if (st != MRA_OK) return st;
  return mra_ws_status(scratch, stream);
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing arrives on,
// with a limit of limit_ns, and records MRA_ETIMEOUT when the wait gives up.
__global__ void k_selftest_wait(unsigned long long limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    const bool ok = mbar_wait_bounded_ns(&bar, 0u, limit_ns);
    *status = ok ? (int)MRA_OK : (int)MRA_ETIMEOUT;
  }
}

MRA_API int mra_selftest_wait_timeout(int32_t limit_us, int32_t* status_out, void* stream) {
  if (limit_us < 1 || limit_us > 2000000 || !ptr_ok(status_out, 4)) return MRA_EINVAL;
  k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((unsigned long long)limit_us * 1000ull,
                                                                  reinterpret_cast<int*>(status_out));
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_selftest_grid_barrier(int32_t limit_us, int32_t* scratch, void* stream) {
  if (limit_us < 1 || limit_us > 2000000 || !ptr_ok(scratch, 16)) return MRA_EINVAL;
  DevInfo di;
  int st = dev_info(&di);
  if (st != MRA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MRA_CUDA_TRY(cudaMemsetAsync(scratch, 0, 4 * sizeof(int32_t), s));
  return launch_selftest_grid_barrier(di.sms, reinterpret_cast<unsigned*>(scratch), reinterpret_cast<int*>(scratch) + 2,
                                      (unsigned long long)limit_us * 1000ull, s);
}

MRA_API int mra_ws_status(void* ws, void* stream) {
  if (!ptr_ok(ws, 256)) return MRA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  const int zero = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(ws, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  return v;
}

}  // extern "C"
