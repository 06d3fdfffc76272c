// Synchronize and Match, rotation-prior fit and relative error on sm_103a.
//
//   pairwise  rel[i][j] = argmax_s Re sum_k C^{ij}_k e^{+2 pi i k s/L},  C^{ij}_k = sum_q conj(y_ikq) y_jkq
//             (= argmin_s sum |y_i - e^{i k theta_s} y_j|^2, Eq. relative_angle_2d_dist)
//   ppm       z <- Hz/||Hz|| then z <- phase(Hz) on H_ij = e^{-2 pi i rel_ij / L}     (Eq. cost_synchronization)
//   match     n*(i) = argmin_{n<P, n != i} ||y_n||^2 - 2 Re <y_i, y_n>, shift_i = phi[n*]
//             (Algorithm Synchronize and Match) -- an (N x 2M) by (2M x P) product with a fused argmin
//   template  shift_j = argmax_s Re sum_k C^{j}_k e^{+2 pi i k s/L},  C^{j}_k = sum_q conj(ref_kq) y_jkq
//             (template matching, Sec. 2.1.1: every image against one reference, O(NLM))
//   fit_prior rho_bar on the window, optional von Mises fit (Algorithm 1 + concentration fit)
//   relerr    min_theta ||R_theta x_hat - x|| / ||x|| (Sec. 2.2)
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "gemm3.cuh"

namespace mra {
namespace {

constexpr int kPairThreads = 128;

// One CTA per pair (i < j) of the first P images.
__global__ void __launch_bounds__(kPairThreads) k_pairwise(const float2* y, int Kp1, int Q, int L, int P, int* rel) {
  extern __shared__ __align__(16) unsigned char psm[];
  float2* tf = reinterpret_cast<float2*>(psm);  // [L] e^{-2 pi i m / L}
  float2* C = tf + L;                           // [Kp1]
  __shared__ float rv[kPairThreads / 32];
  __shared__ int ri[kPairThreads / 32];
  const int i = blockIdx.y, j = blockIdx.x, tid = threadIdx.x;
  if (j < i) return;
  if (j == i) {
    if (tid == 0) rel[(size_t)i * P + i] = 0;
    return;
  }
  const int M = Kp1 * Q;
  for (int m = tid; m < L; m += kPairThreads) {
    float s, c;
    sincospif(2.0f * (float)m / (float)L, &s, &c);
    tf[m] = make_float2(c, -s);
  }
  const float2* yi = y + (size_t)i * M;
  const float2* yj = y + (size_t)j * M;
  for (int k = tid; k < Kp1; k += kPairThreads) {
    float cr = 0.f, ci = 0.f;
    for (int q = 0; q < Q; ++q) {
      const float2 a = yi[k * Q + q], b = yj[k * Q + q];
      cr = fmaf(a.x, b.x, cr); cr = fmaf(a.y, b.y, cr);
      ci = fmaf(a.x, b.y, ci); ci = fmaf(-a.y, b.x, ci);
    }
    C[k] = make_float2(cr, ci);
  }
  __syncthreads();
  float best = -INFINITY;
  int bi = 0x7fffffff;
  for (int l = tid; l < L; l += kPairThreads) {
    float s = 0.f;
    int m = 0;
    for (int k = 0; k < Kp1; ++k) {
      const float2 t = tf[m], c = C[k];  // Re(C e^{+i phi}) with t = e^{-i phi}
      s = fmaf(c.x, t.x, s);
      s = fmaf(c.y, t.y, s);
      m += l;
      if (m >= L) m -= L;
    }
    if (s > best) best = s, bi = l;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
  }
  if ((tid & 31) == 0) rv[tid >> 5] = best, ri[tid >> 5] = bi;
  __syncthreads();
  if (tid == 0) {
    float b = rv[0];
    int idx = ri[0];
    for (int w = 1; w < kPairThreads / 32; ++w)
      if (rv[w] > b || (rv[w] == b && ri[w] < idx)) b = rv[w], idx = ri[w];
    rel[(size_t)i * P + j] = idx;
    rel[(size_t)j * P + i] = (L - idx) % L;
  }
}

// Template matching: a warp per image (grid-stride).  The warp stages its image in shared
// memory with 16-byte loads, lane k forms C_k against the reference held by the CTA (each lane
// starts its walk over q at k mod Q, which spreads the lanes over the banks), and the lanes scan
// the L grid shifts for the largest Re sum_k C_k e^{+2 pi i k s/L} (smallest s among ties), which
// is argmin_s sum |ref - e^{i k theta_s} y_j|^2.  Shifts s and L - s share cos and sin: with
// A = sum C.x cos, B = sum C.y (-sin), the values are A + B at s and A - B at L - s.
constexpr int kTmThreads = 256;
__host__ __device__ inline int tm_even(int v) { return (v + 1) & ~1; }
constexpr int kTmReseed = 8;
__global__ void __launch_bounds__(kTmThreads) k_template_match(const float2* y, const float2* ref, int N, int Kp1,
                                                               int Q, int L, int nwarps, int* shift) {
  extern __shared__ __align__(16) unsigned char tsm[];
  // every image buffer starts on a 16-byte boundary (it is filled with 16-byte stores): offsets in
  // float2 are even (M is even; L and K + 1 are rounded up)
  const int M = Kp1 * Q;
  float2* tf = reinterpret_cast<float2*>(tsm);  // [L] e^{-2 pi i m / L}
  float2* rs = tf + tm_even(L);                 // [M] the reference
  float2* base = rs + M;                        // per warp: [M] image, then [K + 1] C
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int m = tid; m < L; m += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)L, &s, &c);
    tf[m] = make_float2((float)c, (float)-s);
  }
  for (int e = tid; e < M; e += blockDim.x) rs[e] = ref[e];
  __syncthreads();
  if (warp >= nwarps) return;
  float2* img = base + (size_t)warp * (M + tm_even(Kp1));
  float2* C = img + M;
  for (int j = blockIdx.x * nwarps + warp; j < N; j += gridDim.x * nwarps) {
    const float4* src = reinterpret_cast<const float4*>(y + (size_t)j * M);
    float4* dst = reinterpret_cast<float4*>(img);
    for (int e = lane; e < M / 2; e += 32) dst[e] = src[e];
    __syncwarp();
    for (int k = lane; k < Kp1; k += 32) {
      float cr = 0.f, ci = 0.f;
      int q = k % Q;
      for (int qq = 0; qq < Q; ++qq) {
        const float2 a = rs[k * Q + q], b = img[k * Q + q];
        cr = fmaf(a.x, b.x, cr); cr = fmaf(a.y, b.y, cr);
        ci = fmaf(a.x, b.y, ci); ci = fmaf(-a.y, b.x, ci);
        if (++q == Q) q = 0;
      }
      C[k] = make_float2(cr, ci);
    }
    __syncwarp();
    float best = -INFINITY;
    int bi = 0x7fffffff;
    auto take = [&](float v, int l) {
      if (v > best || (v == best && l < bi)) best = v, bi = l;
    };
    // four pairs {l, L - l} per lane at a time (l = lane + 32 (i0 + g)); the twiddle e^{-2 pi i k l / L} steps
    // from k to k + 1 by one complex product with e^{-2 pi i l / L} and is reloaded from the table every
    // kTmReseed rows (bounded rounding drift; table reads of different lanes meet in the same banks)
    const int npair = L / 2 + 1;
    for (int i0 = 0; lane + 32 * i0 < npair; i0 += 4) {
      float A[4], B[4];
      float2 t[4], w[4];
      int l[4], m[4], m8[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        l[g] = min(lane + 32 * (i0 + g), npair - 1);
        w[g] = tf[l[g]];
        m[g] = 0;
        m8[g] = (int)(((long long)kTmReseed * l[g]) % L);
        A[g] = 0.f, B[g] = 0.f;
      }
      for (int k0 = 0; k0 < Kp1; k0 += kTmReseed) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          t[g] = tf[m[g]];
          m[g] += m8[g];
          if (m[g] >= L) m[g] -= L;
        }
        const int k1 = min(k0 + kTmReseed, Kp1);
        for (int k = k0; k < k1; ++k) {
          const float2 c = C[k];  // Re(C e^{+i phi}) = A + B with t = e^{-i phi}
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            A[g] = fmaf(c.x, t[g].x, A[g]);
            B[g] = fmaf(c.y, t[g].y, B[g]);
            t[g] = cmul(t[g], w[g]);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int lg = lane + 32 * (i0 + g);
        if (lg < npair) {
          take(A[g] + B[g], lg);
          if (lg > 0 && 2 * lg != L) take(A[g] - B[g], L - lg);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
    }
    if (lane == 0) shift[j] = bi < L ? bi : 0;  // bi >= L only if every value is NaN
    __syncwarp();  // the image and C buffers are rewritten for the next image
  }
}

// Projected power method, one CTA: a group of g lanes (a power of two, g <= 32)
// forms (Hz)_i for each row i, lanes striding over j, then sums with log2(g)
// shuffles.  rel is staged in shared memory as int16 when it fits.
constexpr int kPpmThreads = 1024;
__global__ void __launch_bounds__(kPpmThreads) k_ppm(int L, int P, const int* rel, int n_power, int n_ppm, int* phi,
                                                     int stage, int g) {
  extern __shared__ __align__(16) unsigned char zsm[];
  float2* tf = reinterpret_cast<float2*>(zsm);  // [L]
  float2* z = tf + L;                           // [P]
  float2* zn = z + P;                           // [P]
  float2* hs = zn + P;                           // [P][P] H when stage == 2
  short* rs = reinterpret_cast<short*>(zn + P);  // [P][P] twiddle indices when stage == 1
  __shared__ float red[33];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows_per_pass = kPpmThreads / g;
  const int sub = tid % g, row0 = tid / g;
  for (int m = tid; m < L; m += kPpmThreads) {
    float s, c;
    sincospif(2.0f * (float)m / (float)L, &s, &c);
    tf[m] = make_float2(c, -s);
  }
  for (int i = tid; i < P; i += kPpmThreads) z[i] = make_float2(1.f, 0.f);
  __syncthreads();
  if (stage) {
    for (int e = tid; e < P * P; e += kPpmThreads) {
      int m = rel[e] % L;
      if (m < 0) m += L;
      if (stage == 2) hs[e] = tf[m];
      else rs[e] = (short)m;
    }
  }
  __syncthreads();
  const int total = n_power + n_ppm;
  for (int it = 0; it < total; ++it) {
    const bool power = it < n_power;
    float part = 0.f;
    for (int i0 = 0; i0 < P; i0 += rows_per_pass) {
      const int i = i0 + row0;
      float vr = 0.f, vi = 0.f;
      if (i < P) {
#pragma unroll 4
        for (int jj = sub; jj < P; jj += g) {
          float2 h;
          if (stage == 2) {
            h = hs[i * P + jj];
          } else {
            int m;
            if (stage == 1) {
              m = rs[i * P + jj];
            } else {
              m = rel[(size_t)i * P + jj] % L;
              if (m < 0) m += L;
            }
            h = tf[m];
          }
          const float2 zz = z[jj];
          vr = fmaf(h.x, zz.x, fmaf(-h.y, zz.y, vr));
          vi = fmaf(h.x, zz.y, fmaf(h.y, zz.x, vi));
        }
      }
      for (int o = 1; o < g; o <<= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (i < P && sub == 0) {
        if (power) {
          zn[i] = make_float2(vr, vi);
          part += vr * vr + vi * vi;
        } else {
          const float a = sqrtf(vr * vr + vi * vi);
          zn[i] = a > 0.f ? make_float2(vr / a, vi / a) : make_float2(1.f, 0.f);
        }
      }
    }
    if (power) {
      part = warp_sum(part);
      if (lane == 0) red[warp] = part;
      __syncthreads();
      if (warp == 0) {
        float t = red[lane];
        t = warp_sum(t);
        if (lane == 0) red[32] = t > 0.f ? rsqrtf(t) : 1.f;
      }
    }
    __syncthreads();
    const float inv = power ? red[32] : 1.f;
    for (int i = tid; i < P; i += kPpmThreads) {
      const float2 v = zn[i];
      z[i] = power ? make_float2(v.x * inv, v.y * inv) : v;
    }
    __syncthreads();
  }
  for (int i = tid; i < P; i += kPpmThreads) {
    const float2 z0 = z[0], zi = z[i];
    const float wr = zi.x * z0.x + zi.y * z0.y, wi = zi.y * z0.x - zi.x * z0.y;  // z_i conj(z_0)
    const float ang = atan2f(wi, wr);
    int sv = (int)floorf(ang * (float)L / (2.0f * (float)kPi) + 0.5f);
    sv %= L;
    if (sv < 0) sv += L;
    phi[i] = (i == 0) ? 0 : sv;
  }
}

__global__ void k_refnorm(const float* y, int D, int P, float* nrm) {
  const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (n >= P) return;
  const float* r = y + (size_t)n * D;
  float s = 0.f;
  for (int d = lane; d < D; d += 32) s = fmaf(r[d], r[d], s);
  s = warp_sum(s);
  if (lane == 0) nrm[n] = s;
}

// Matching: 128 queries x 128 references per tile, 16 real coordinates per step,
// 8 x 8 outputs per thread; score = ||y_n||^2 - 2 <y_i, y_n>, running argmin per query.
// The next step's coordinates are fetched into registers while the current step
// computes from the other shared-memory buffer.  Lanes run over query groups and warps
// over reference groups, so that a warp whose reference columns all lie beyond P (the
// second half of the last tile when P is not a multiple of 128) skips those products.
constexpr int kMT = 128, kKC = 16;
__global__ void __launch_bounds__(256) k_match(const float* y, int N, int D, int P, const float* nrm, const int* phi,
                                               int* shift_out) {
  __shared__ __align__(16) float As[2][kKC][kMT + 4];
  __shared__ __align__(16) float Bs[2][kKC][kMT + 4];
  const int tid = threadIdx.x;
  const int tq = tid & 15, tr = tid >> 4;  // a warp holds tr = 2w, 2w + 1
  const int q0 = blockIdx.x * kMT;
  const int lrow = tid >> 1, lh = (tid & 1) * 8;  // loader: row and 8-coordinate half of a step
  float bestv[8];
  int besti[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) bestv[u] = INFINITY, besti[u] = 0x7fffffff;

  for (int r0 = 0; r0 < P; r0 += kMT) {
    const int qi = q0 + lrow, ri = r0 + lrow;
    const float* qa = y + (size_t)min(qi, N - 1) * D;
    const float* ra = y + (size_t)min(ri, P - 1) * D;
    float4 pa[2], pb[2];
    auto fetch = [&](int kc) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int d = kc + lh + 4 * h;
        const bool in = d < D;
        pa[h] = (qi < N && in) ? *reinterpret_cast<const float4*>(qa + d) : make_float4(0.f, 0.f, 0.f, 0.f);
        pb[h] = (ri < P && in) ? *reinterpret_cast<const float4*>(ra + d) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = lh + 4 * h;
        As[buf][e][lrow] = pa[h].x; As[buf][e + 1][lrow] = pa[h].y;
        As[buf][e + 2][lrow] = pa[h].z; As[buf][e + 3][lrow] = pa[h].w;
        Bs[buf][e][lrow] = pb[h].x; Bs[buf][e + 1][lrow] = pb[h].y;
        Bs[buf][e + 2][lrow] = pb[h].z; Bs[buf][e + 3][lrow] = pb[h].w;
      }
    };
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
    // reference columns of this warp: r0 + 8w .. r0 + 8w + 7 in each half (warp-uniform tests)
    const int wc = r0 + 8 * (tid >> 5);
    const bool lo_on = wc < P, hi_on = wc + 64 < P;
    fetch(0);
    int buf = 0;
    for (int kc = 0; kc < D; kc += kKC, buf ^= 1) {
      stash(buf);
      __syncthreads();
      if (kc + kKC < D) fetch(kc + kKC);
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tq * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tq * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tr * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tr * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        if (lo_on) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        if (hi_on) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 4; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
      }
    }
    __syncthreads();  // the buffers are refilled by the next reference tile
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + (u < 4 ? tq * 4 + u : 64 + tq * 4 + (u - 4));
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const int n = r0 + (v < 4 ? tr * 4 + v : 64 + tr * 4 + (v - 4));
        if (n < P && n != q) {
          const float sc = nrm[n] - 2.f * acc[u][v];
          if (sc < bestv[u] || (sc == bestv[u] && n < besti[u])) bestv[u] = sc, besti[u] = n;
        }
      }
    }
  }
  // reduce over the 16 threads (one per tr, in different warps) that share each query, through
  // shared memory (the tile buffers are free after the last barrier of the reference loop)
  float* rv = &As[0][0][0];                      // [16][kMT]
  int* ri = reinterpret_cast<int*>(&Bs[0][0][0]);  // [16][kMT]
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int ql = u < 4 ? tq * 4 + u : 64 + tq * 4 + (u - 4);
    rv[tr * kMT + ql] = bestv[u];
    ri[tr * kMT + ql] = besti[u];
  }
  __syncthreads();
  if (tid < kMT) {
    float bv = rv[tid];
    int bi = ri[tid];
    for (int t = 1; t < 16; ++t) {
      const float ov = rv[t * kMT + tid];
      const int oi = ri[t * kMT + tid];
      if (ov < bv || (ov == bv && oi < bi)) bv = ov, bi = oi;
    }
    const int q = q0 + tid;
    if (q < N) shift_out[q] = (bi < P) ? phi[bi] : 0;
  }
}

// --- von Mises: A(kappa) = I_1(kappa)/I_0(kappa)
// kappa < 50: backward recurrence of r_n = I_{n+1}/I_n = 1/(2(n+1)/kappa + r_{n+1}) from a deep start;
// kappa >= 50: large-argument expansion I_nu(x) ~ e^x/sqrt(2 pi x) sum_k (-1)^k a_k(nu)/x^k,
//              a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (k! 8^k).
__device__ double vm_A(double kappa) {
  if (kappa <= 0.0) return 0.0;
  if (kappa < 50.0) {
    const int n0 = (int)(2.0 * kappa) + 60;
    double r = 0.0;
    for (int n = n0; n >= 0; --n) r = 1.0 / (2.0 * (double)(n + 1) / kappa + r);
    return r;
  }
  double s0 = 1.0, s1 = 1.0, t0 = 1.0, t1 = 1.0;
  for (int k = 1; k <= 12; ++k) {
    const double f = (double)(2 * k - 1) * (double)(2 * k - 1);
    t0 *= -(0.0 - f) / ((double)k * 8.0 * kappa);
    t1 *= -(4.0 - f) / ((double)k * 8.0 * kappa);
    s0 += t0;
    s1 += t1;
  }
  return s1 / s0;
}

// Grid bin of window position i: (l0 + i) mod L on the grid, else the bin nearest to step (l0 + i).
__device__ inline int prior_bin(int L, int l0, int i, double step) {
  long long b;
  if (step == 1.0)
    b = (long long)l0 + i;
  else
    b = (long long)floor(__dadd_rn(__dmul_rn(step, (double)(l0 + i)), 0.5));  // rounded product, then the add
  b %= L;
  return (int)(b < 0 ? b + L : b);
}

__global__ void k_fit_prior(int L, int Lw, int l0, double step, const int* counts, int kind, double* log_prior,
                            double* kappa_out) {
  __shared__ double red[32];
  __shared__ double bc[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  auto bsum = [&](double v) {
    v = warp_sum_d(v);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) t += red[w];
    return t;
  };
  double tot = 0.0, mc = 0.0;
  for (int s = tid; s < L; s += nt) {
    tot += (double)counts[s];
    mc += (double)counts[s] * cospi(2.0 * (double)s / (double)L);
  }
  tot = bsum(tot);
  mc = bsum(mc);
  if (kind == 0) {
    double wsum = 0.0;
    for (int i = tid; i < Lw; i += nt) wsum += (double)counts[prior_bin(L, l0, i, step)];
    wsum = bsum(wsum);
    for (int i = tid; i < Lw; i += nt) log_prior[i] = log((double)counts[prior_bin(L, l0, i, step)] / wsum);
    if (tid == 0 && kappa_out) *kappa_out = 0.0;
    return;
  }
  if (tid == 0) {
    const double target = mc / tot;
    double kap = 0.0;
    if (target > 0.0) {
      double lo = 0.0, hi = 1.0;
      while (vm_A(hi) < target && hi < 1e12) hi *= 2.0;
      for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (vm_A(mid) < target) lo = mid; else hi = mid;
      }
      kap = 0.5 * (lo + hi);
    }
    bc[0] = kap;
  }
  __syncthreads();
  const double kap = bc[0];
  double mx = -INFINITY;
  for (int i = tid; i < Lw; i += nt) mx = fmax(mx, kap * cospi(2.0 * step * (double)(l0 + i) / (double)L));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = -INFINITY;
    for (int w = 0; w < (nt + 31) / 32; ++w) m = fmax(m, red[w]);
    bc[1] = m;
  }
  __syncthreads();
  const double m = bc[1];
  double z = 0.0;
  for (int i = tid; i < Lw; i += nt) z += exp(kap * cospi(2.0 * step * (double)(l0 + i) / (double)L) - m);
  z = bsum(z);
  const double lz = m + log(z);
  for (int i = tid; i < Lw; i += nt) log_prior[i] = kap * cospi(2.0 * step * (double)(l0 + i) / (double)L) - lz;
  if (tid == 0 && kappa_out) *kappa_out = kap;
}

// Relative error: FP32 scan of 4096 angles, FP64 golden-section refinement (one CTA).
__global__ void k_relerr(int Kp1, int Q, const double2* xh, const double2* x, double* err) {
  extern __shared__ __align__(16) unsigned char rsm[];
  double2* g = reinterpret_cast<double2*>(rsm);  // [Kp1]
  __shared__ double red[32];
  __shared__ float fv[32];
  __shared__ int fi[32];
  __shared__ double AB[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  double A = 0.0, Bn = 0.0;
  for (int e = tid; e < Kp1 * Q; e += nt) {
    const double wk = (e / Q) > 0 ? 2.0 : 1.0;
    A += wk * (xh[e].x * xh[e].x + xh[e].y * xh[e].y);
    Bn += wk * (x[e].x * x[e].x + x[e].y * x[e].y);
  }
  A = warp_sum_d(A);
  Bn = warp_sum_d(Bn);
  if ((tid & 31) == 0) red[tid >> 5] = A;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) t += red[w];
    AB[0] = t;
  }
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = Bn;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) t += red[w];
    AB[1] = t;
  }
  for (int k = tid; k < Kp1; k += nt) {  // g_k = w_k sum_q xh_kq conj(x_kq)
    const double wk = k > 0 ? 2.0 : 1.0;
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < Q; ++q) {
      const double2 a = xh[k * Q + q], b = x[k * Q + q];
      s.x += a.x * b.x + a.y * b.y;
      s.y += a.y * b.x - a.x * b.y;
    }
    g[k] = make_double2(wk * s.x, wk * s.y);
  }
  __syncthreads();
  // f(theta) = A + B - 2 Re sum_k g_k e^{-i k theta}; maximise h(theta) = Re sum_k g_k e^{-i k theta}
  const int NG = 4096;
  float best = -INFINITY;
  int bi = 0;
  for (int t = tid; t < NG; t += nt) {
    float s = 0.f;
    for (int k = 0; k < Kp1; ++k) {
      float sn, cs;
      sincospif(2.0f * (float)(((long long)k * t) % NG) / (float)NG, &sn, &cs);
      s += (float)g[k].x * cs + (float)g[k].y * sn;
    }
    if (s > best) best = s, bi = t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
  }
  if ((tid & 31) == 0) fv[tid >> 5] = best, fi[tid >> 5] = bi;
  __syncthreads();
  if (tid == 0) {
    float b = fv[0];
    int idx = fi[0];
    for (int w = 1; w < (nt + 31) / 32; ++w)
      if (fv[w] > b || (fv[w] == b && fi[w] < idx)) b = fv[w], idx = fi[w];
    auto h = [&](double th) {
      double sn, cs;
      sincos(th, &sn, &cs);
      double er = 1.0, ei = 0.0, s = 0.0;  // e^{-i k th} by recurrence
      for (int k = 0; k < Kp1; ++k) {
        s += g[k].x * er - g[k].y * ei;
        const double nr = er * cs + ei * sn, ni = ei * cs - er * sn;
        er = nr;
        ei = ni;
      }
      return s;
    };
    const double step = 2.0 * kPi / NG;
    double lo = idx * step - step, hi = idx * step + step;
    const double gr = 0.6180339887498949;
    double c1 = hi - gr * (hi - lo), c2 = lo + gr * (hi - lo);
    double h1 = h(c1), h2 = h(c2);
    for (int it = 0; it < 80; ++it) {
      if (h1 > h2) { hi = c2; c2 = c1; h2 = h1; c1 = hi - gr * (hi - lo); h1 = h(c1); }
      else { lo = c1; c1 = c2; h1 = h2; c2 = lo + gr * (hi - lo); h2 = h(c2); }
    }
    const double hbest = fmax(fmax(h1, h2), h(idx * step));
    const double f = fmax(AB[0] + AB[1] - 2.0 * hbest, 0.0);
    *err = sqrt(f) / sqrt(AB[1]);
  }
}

bool ok_ptr(const void* p, size_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_sync_dims(const mra_dims* d, int P) {
  if (!d || d->N < 1 || d->K < 0 || d->Q < 1 || d->L < 1) return MRA_EINVAL;
  if (P < 1 || P > d->N) return MRA_EINVAL;
  if (((long long)(d->K + 1) * d->Q) % 2 != 0) return MRA_EINVAL;
  return MRA_OK;
}

// Sync workspace: a status word (the bounded waits of the tensor-core match), the relative rotations,
// the synchronized rotations, the references' norms and, for P <= 256, the references packed as the
// tensor-core GEMM's B operand (coordinates as K).
struct SyncLayout {
  size_t status, rel, phi, nrm, bpack, total;
  int KB, brows;  // K blocks of the packed references, and their rows (P rounded up to 16)
};
bool match_on_tc(int P) { return P <= kG3Cols; }
SyncLayout sync_layout(int P, int D) {
  SyncLayout s;
  size_t o = 0;
  s.status = o; o = 256;
  s.rel = o; o = align256(o + sizeof(int) * (size_t)P * P);
  s.phi = o; o = align256(o + sizeof(int) * (size_t)P);
  s.nrm = o; o = align256(o + sizeof(float) * (size_t)P);
  s.KB = (D + kG3KB - 1) / kG3KB;
  s.brows = (P + 15) / 16 * 16;
  s.bpack = o; o = align256(o + (match_on_tc(P) ? (size_t)s.KB * 3 * s.brows * kG3KB * 2 : 0));
  s.total = o;
  return s;
}

}  // namespace
}  // namespace mra

using namespace mra;

extern "C" {

MRA_API size_t mra_sync_workspace_bytes(const mra_dims* d, int32_t P) {
  if (check_sync_dims(d, P) != MRA_OK) return 0;
  return sync_layout(P, 2 * (d->K + 1) * d->Q).total;
}

MRA_API int mra_sync_pairwise(const mra_dims* d, const float* y, int32_t P, int32_t* rel_out, void* stream) {
  if (check_sync_dims(d, P) != MRA_OK || !ok_ptr(y, 16) || !ok_ptr(rel_out, 4)) return MRA_EINVAL;
  if (d->L > 8192 || d->K + 1 > 4096) return MRA_EINVAL;
  const int smem = (d->L + d->K + 1) * 8;
  if (smem > 48 * 1024 && raise_smem_limit(reinterpret_cast<const void*>(k_pairwise), smem) != MRA_OK)
    return MRA_ECUDA;
  k_pairwise<<<dim3(P, P), kPairThreads, smem, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float2*>(y), d->K + 1, d->Q, d->L, P, rel_out);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_template_match(const mra_dims* d, const float* y, const float* ref, int32_t* shift_out,
                               void* stream) {
  if (check_sync_dims(d, 1) != MRA_OK || !ok_ptr(y, 16) || !ok_ptr(ref, 16) || !ok_ptr(shift_out, 4))
    return MRA_EINVAL;
  if (d->L > 8192) return MRA_EINVAL;
  DevInfo di;
  if (dev_info(&di) != MRA_OK) return MRA_ECUDA;
  const int Kp1 = d->K + 1, M = Kp1 * d->Q;
  const int fixed = (tm_even(d->L) + M) * 8, per_warp = (M + tm_even(Kp1)) * 8;
  const int budget = std::min(di.max_smem_optin, 96 * 1024);  // room for two CTAs per SM
  const int nwarps = std::min(kTmThreads / 32, (budget - fixed) / per_warp);
  if (nwarps < 1) return MRA_EINVAL;
  const int smem = fixed + nwarps * per_warp;
  if (smem > 48 * 1024 &&
      raise_smem_limit(reinterpret_cast<const void*>(k_template_match), smem) != MRA_OK)
    return MRA_ECUDA;
  const long long need = ((long long)d->N + nwarps - 1) / nwarps;
  const int grid = (int)std::min<long long>(need, (long long)di.sms * 8);
  k_template_match<<<grid, kTmThreads, smem, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float2*>(y), reinterpret_cast<const float2*>(ref), d->N, Kp1, d->Q, d->L, nwarps,
      shift_out);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_sync_ppm(int32_t L, int32_t P, const int32_t* rel, int32_t n_power, int32_t n_ppm, int32_t* phi_out,
                         void* stream) {
  if (L < 1 || L > 8192 || P < 1 || P > 1024 || n_power < 0 || n_ppm < 0 || !ok_ptr(rel, 4) || !ok_ptr(phi_out, 4))
    return MRA_EINVAL;
  const int base = (L + 2 * P) * 8;
  const int stage = (base + P * P * 8 <= 200 * 1024) ? 2 : (base + P * P * 2 <= 200 * 1024) ? 1 : 0;
  const int smem = base + (stage == 2 ? P * P * 8 : stage == 1 ? P * P * 2 : 0);
  if (smem > 48 * 1024 && raise_smem_limit(reinterpret_cast<const void*>(k_ppm), smem) != MRA_OK) return MRA_ECUDA;
  int g = 32;  // lanes per row: the largest power of two with g * P <= 1024
  while (g > 1 && g * P > kPpmThreads) g >>= 1;
  k_ppm<<<1, kPpmThreads, smem, static_cast<cudaStream_t>(stream)>>>(L, P, rel, n_power, n_ppm, phi_out, stage, g);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_sync_match(const mra_dims* d, const float* y, int32_t P, const int32_t* phi, int32_t* shift_out,
                           void* ws, size_t ws_bytes, void* stream) {
  if (check_sync_dims(d, P) != MRA_OK || !ok_ptr(y, 16) || !ok_ptr(phi, 4) || !ok_ptr(shift_out, 4) ||
      !ok_ptr(ws, 256))
    return MRA_EINVAL;
  const int D = 2 * (d->K + 1) * d->Q;
  const SyncLayout sl = sync_layout(P, D);
  if (ws_bytes < sl.total) return MRA_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = static_cast<unsigned char*>(ws);
  float* nrm = reinterpret_cast<float*>(base + sl.nrm);
  k_refnorm<<<(P + 7) / 8, 256, 0, s>>>(y, D, P, nrm);
  if (match_on_tc(P)) {
    // score_in = ||y_n||^2 - 2 <y_i, y_n> from the tensor-core GEMM of the images with the P references
    DevInfo di;
    if (dev_info(&di) != MRA_OK) return MRA_ECUDA;
    if (raise_smem_limit(reinterpret_cast<const void*>(k_gemm3<1>), kG3Smem) != MRA_OK) return MRA_ECUDA;
    k_gemm3_pack<<<1024, 256, 0, s>>>(y, D, 1, P, D, 1, sl.KB, sl.brows, base + sl.bpack);
    Gemm3Args g{};
    g.A = y;
    g.lda = D;
    g.rows = d->N;
    g.K = D;
    g.Bp = base + sl.bpack;
    g.NT = 1;
    g.KB = sl.KB;
    g.cols = P;
    g.nprod = 6;
    g.brows = sl.brows;
    g.rn = nrm;
    g.phi = phi;
    g.out = shift_out;
    g.status = reinterpret_cast<int*>(base + sl.status);
    const int items = (d->N + kG3Rows - 1) / kG3Rows;
    k_gemm3<1><<<std::min(items, di.sms), kG3Threads, kG3Smem, s>>>(g);
  } else {
    k_match<<<(d->N + kMT - 1) / kMT, 256, 0, s>>>(y, d->N, D, P, nrm, phi, shift_out);
  }
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_sync(const mra_dims* d, const float* y, int32_t P, int32_t n_power, int32_t n_ppm, int32_t* shift_out,
                     void* ws, size_t ws_bytes, void* stream) {
  if (check_sync_dims(d, P) != MRA_OK || !ok_ptr(ws, 256)) return MRA_EINVAL;
  const SyncLayout sl = sync_layout(P, 2 * (d->K + 1) * d->Q);
  if (ws_bytes < sl.total) return MRA_EWORKSPACE;
  unsigned char* base = static_cast<unsigned char*>(ws);
  int* rel = reinterpret_cast<int*>(base + sl.rel);
  int* phi = reinterpret_cast<int*>(base + sl.phi);
  int st = mra_sync_pairwise(d, y, P, rel, stream);
  if (st != MRA_OK) return st;
  if ((st = mra_sync_ppm(d->L, P, rel, n_power, n_ppm, phi, stream)) != MRA_OK) return st;
  return mra_sync_match(d, y, P, phi, shift_out, ws, ws_bytes, stream);
}

MRA_API int mra_fit_prior(int32_t L, int32_t Lw, int32_t l0, double step, const int32_t* counts, int32_t kind,
                          double* log_prior_out, double* kappa_out, void* stream) {
  if (step == 0.0) step = 1.0;
  if (L < 1 || (kind != 0 && kind != 1) || !ok_ptr(counts, 4) || !ok_ptr(log_prior_out, 8)) return MRA_EINVAL;
  if (!window_ok(L, Lw, l0, step)) return MRA_EINVAL;
  if (kappa_out && !ok_ptr(kappa_out, 8)) return MRA_EINVAL;
  k_fit_prior<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(L, Lw, l0, step, counts, kind, log_prior_out,
                                                                kappa_out);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_relerr(int32_t K, int32_t Q, const double* x_hat, const double* x, double* err_out, void* stream) {
  if (K < 0 || Q < 1 || !ok_ptr(x_hat, 16) || !ok_ptr(x, 16) || !ok_ptr(err_out, 8)) return MRA_EINVAL;
  if ((K + 1) * 16 > 40 * 1024) return MRA_EINVAL;
  k_relerr<<<1, 256, (K + 1) * 16, static_cast<cudaStream_t>(stream)>>>(
      K + 1, Q, reinterpret_cast<const double2*>(x_hat), reinterpret_cast<const double2*>(x), err_out);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

}  // extern "C"
