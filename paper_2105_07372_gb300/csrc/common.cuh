// Shared device helpers and the workspace layout of libmra (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mra.h"

#define MRA_CUDA_TRY(expr)                        \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return MRA_ECUDA;      \
  } while (0)

namespace mra {

constexpr int kSweepThreads = 256;
constexpr int kSweepWarps = kSweepThreads / 32;
constexpr double kPi = 3.141592653589793238462643383279502884;
// Bounded device waits give up after this many nanoseconds and report MRA_ETIMEOUT.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------- small math
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj_b(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// Two complex values of y at float4 index f of an image: FP32 (YF = 0), or the BF16
// hi/lo split (YF = 1) whose 16-byte group f holds bf16 hi of (re, im, re, im) and then
// bf16 lo of the same four values; hi + lo is exact in FP32.
template <int YF>
__device__ __forceinline__ float4 load_y4(const float4* img, int f) {
  if constexpr (YF == 0) {
    return img[f];
  } else {
    const uint4 v = reinterpret_cast<const uint4*>(img)[f];
    const float2 h0 = make_float2(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u));
    const float2 h1 = make_float2(__uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    const float2 l0 = make_float2(__uint_as_float(v.z << 16), __uint_as_float(v.z & 0xffff0000u));
    const float2 l1 = make_float2(__uint_as_float(v.w << 16), __uint_as_float(v.w & 0xffff0000u));
    const float2 a = __fadd2_rn(h0, l0), b = __fadd2_rn(h1, l1);
    return make_float4(a.x, a.y, b.x, b.y);
  }
}

// e^{-i t sgn(dr)} from a distance-unit table entry (cos t - 1, -sin t) taken at |dr|.
__device__ __forceinline__ float2 td_rot(float2 t, int dr) { return make_float2(1.f + t.x, dr >= 0 ? t.y : -t.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- mbarrier + bulk copy (TMA)
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Invalidate an mbarrier whose phases are all complete, before its memory is used otherwise.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// As mbar_try_wait, but the thread may be suspended (issuing nothing) until the phase
// completes or about hint_ns nanoseconds have passed.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
constexpr uint32_t kSuspendHintNs = 50000;  // one suspension; the time limit is checked between them
// Wait for the phase with the given parity; false if it did not complete within kWaitLimitNs.
// Waiting threads are suspended rather than spinning, so they take no issue slots from the
// warps that have work.
__device__ __forceinline__ bool mbar_wait_bounded_ns(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_suspend(bar, parity, kSuspendHintNs)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  return mbar_wait_bounded_ns(bar, parity, kWaitLimitNs);
}
// One-dimensional bulk copy global -> shared, completion counted on bar (bytes, addresses: multiples of 16).
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------- workspace
// Control words at the start of every workspace.
struct Ctrl {
  int status;  // MRA_OK or MRA_ETIMEOUT, set by kernels
  int done;    // em_run: converged flag, makes the remaining kernels of a graph return at entry
  int iter;    // em_run: iterations performed
  unsigned sched[2];  // wide-window warp sweep: next image and finished warps (zero between launches)
  unsigned fin;       // finalize: CTAs done with their columns (zero between launches)
  int pad[58];
};

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
constexpr int kUnitChunk = 20;  // mirror units per warp chunk: 4 lanes x 5 units

// Offsets (bytes) of every array in the EM workspace; identical on host and device.
struct EmLayout {
  int G;        // persistent grid of the sweep
  int M, Kp1, Lw, L;
  int twp;      // padded row pitch (in complex) of the window twiddle table
  int kp4;      // K+1 rounded up to a multiple of 4 (rows of the table)
  int cols;     // 2M + Lw + 2 reduced columns
  int nup;      // mirror units padded to a multiple of kUnitChunk
  size_t ctrl, tf32, tf64, tw, tw64, x32, x64, inv_den, logrho32, rho64, rhobar64, units, tu, td, part, tot;
  size_t tcb, cbuf, wbuf;  // split sweep only (zero-sized otherwise)
  size_t total;
};

__host__ __device__ inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
// The split sweep's extra workspace (correlation and weight buffers, the B operand) exists for
// windows it can take: wider than 64 rotations, at most 1024 (two passes of 512 tensor-memory
// columns beyond 512), K+1 <= 48.
__host__ __device__ inline bool split_possible(int Kp1, int Q, int Lw) {
  return Lw > 64 && Lw <= 1024 && Kp1 <= 48 && Q % 8 == 0 && Q / 8 <= 4;
}

inline EmLayout em_layout(int N, int K, int Q, int L, int Lw, int G) {
  EmLayout l{};
  l.G = G;
  l.Kp1 = K + 1;
  l.M = (K + 1) * Q;
  l.Lw = Lw;
  l.L = L;
  l.twp = (Lw + 3) & ~3;
  l.kp4 = (K + 1 + 3) & ~3;
  l.cols = 2 * l.M + Lw + 2;
  l.nup = round_up(Lw, kUnitChunk);  // the unit count never exceeds Lw
  size_t o = 0;
  l.ctrl = o;      o = align256(o + sizeof(Ctrl));
  l.tf32 = o;      o = align256(o + sizeof(float2) * L);
  l.tf64 = o;      o = align256(o + sizeof(double2) * L);
  l.tw = o;        o = align256(o + sizeof(float2) * (size_t)l.kp4 * l.twp);
  l.tw64 = o;      o = align256(o + sizeof(double2) * (size_t)l.kp4 * l.twp);
  l.x32 = o;       o = align256(o + sizeof(float2) * l.M);
  l.x64 = o;       o = align256(o + sizeof(double2) * l.M);
  l.inv_den = o;   o = align256(o + sizeof(double) * l.M);
  l.logrho32 = o;  o = align256(o + sizeof(float) * Lw);
  l.rho64 = o;     o = align256(o + sizeof(double) * Lw);
  l.rhobar64 = o;  o = align256(o + sizeof(double) * Lw);
  l.units = o;     o = align256(o + sizeof(int2) * l.nup);
  l.tu = o;        o = align256(o + sizeof(float2) * (size_t)l.Kp1 * l.nup);
  l.td = o;        o = align256(o + sizeof(float2) * (size_t)l.Kp1 * (size_t)(Lw > L / 2 + 1 ? Lw : L / 2 + 1));
  l.part = o;      o = align256(o + sizeof(double) * (size_t)l.cols * G);
  l.tot = o;       o = align256(o + sizeof(double) * (l.cols + 8));
  const bool split = split_possible(l.Kp1, Q, Lw);
  const size_t ka = (size_t)((2 * ((l.Kp1 + 3) / 4 * 4) + 15) / 16 * 16), np = (size_t)((Lw + 15) / 16 * 16);
  l.tcb = o;       o = align256(o + (split ? np * ka * 2 : 0));
  l.cbuf = o;      o = align256(o + (split ? sizeof(float2) * (size_t)N * l.Kp1 : 0));
  l.wbuf = o;      o = align256(o + (split ? sizeof(float2) * (size_t)N * l.Kp1 : 0));
  l.total = o;
  return l;
}

// Arguments of the warp-per-image sweep (sweep_impl.cuh).
struct SweepV2Args {
  const float2* y;
  const int* shift;
  int N, Kp1, M, L, Lw, NU, NUP;
  int nwarps;      // active warps per CTA
  int slot_bytes;  // bytes per ring slot
  int sp;          // per-warp row pitch (floats) of the s/w and W[l] buffers
  int off_ring, off_x, off_tu, off_tf, off_lr, off_units, off_s, off_wl;
  int cbp;         // lean sweep: per-warp buffer pitch (float2) for c_k and the window's values
  float two_beta;
  int align_only;  // 1: weights are 1 at offset 0 (align and average)
  int wrap;        // 1: the window is the whole grid circle (Lw == L), distances wrap
  int l0m;         // l0 mod L (grid windows)
  int nd;          // distance units in td: L/2 + 1 when wrapping, else Lw
  const float2* x32;
  const float2* tu;    // [Kp1][NUP] e^{-i k theta} of each mirror unit's first offset
  const int2* units;   // [NUP] window indices (a, b), b = -1 for a unit without mirror
  const float2* td;    // [Kp1][nd] (cos t - 1, -sin t), t = 2 pi k d step / L (global)
  const float2* tw;    // dense window only (else null): [Kp1][twp] e^{-i k theta_{l0+i}} (global)
  int twp;
  const float2* tf32;
  const float* logrho32;
  double* part;
  int G;
  float* w_out;
  Ctrl* ctrl;
};
struct SweepV2Launch {
  void (*fn)(const SweepV2Args);
  int threads;
};
// ipw: images each warp carries at once (only 1 is built); lwc: for a window of one unit
// chunk, lane-strided passes over it fixed at compile time (1 for Lw <= 32, 2 for Lw <= 64),
// else 0 (any window).
SweepV2Launch sweep_v2_q1(int MR, int ipw, int lwc);
SweepV2Launch sweep_v2_q2(int MR, int ipw, int lwc);
SweepV2Launch sweep_v2_q3(int MR, int ipw, int lwc);
SweepV2Launch sweep_v2_q4(int MR, int ipw, int lwc);
// Lean warp sweep (sweep5_impl.cuh): grid windows of at most 32 mirror units (unit pitch nup
// 20 or 40), the same arguments and tables as the warp sweep plus cbp.
SweepV2Launch sweep_v5_q1(int MR, int nup);
SweepV2Launch sweep_v5_q2(int MR, int nup);
SweepV2Launch sweep_v5_q3(int MR, int nup);
SweepV2Launch sweep_v5_q4(int MR, int nup);

// Arguments of the paired-warp sweep (sweep6_impl.cuh): grid windows of at most 32 mirror units,
// two warps per image, the tables of the warp sweep (units, tu, td).
struct SweepV6Args {
  const float2* y;
  const int* shift;
  int N, K, M, L, Lw, NU;
  int ns;          // ring slots per warp pair
  int slot_bytes;  // bytes per ring slot
  int sp;          // pitch (floats) of the per-warp window buffers
  int off_bar, off_ring, off_tab, off_tf, off_lr, off_units, off_cb, off_xp, off_xq, off_pv, off_sb, off_wl;
  float two_beta;
  int l0m;         // l0 mod L
  int nd;          // distance units in td (Lw)
  int nup;         // pitch of tu
  const float2* x32;
  const float2* tu;    // [Kp1][nup] e^{-i k theta} of each mirror unit's first offset
  const int2* units;   // [nup] window indices (a, b), b = -1 for a unit without mirror
  const float2* td;    // [Kp1][nd] (cos t - 1, -sin t), t = 2 pi k d / L
  const float2* tf32;
  const float* logrho32;
  double* part;
  int G;
  float* w_out;
  Ctrl* ctrl;
};
struct SweepV6Launch {
  void (*fn)(const SweepV6Args);
  int threads;
};
// QV = float4 per lane per row (Q / 8); MR = rows per quad and warp (K <= 16 MR); instances with
// MR x QV <= 6.
SweepV6Launch sweep_v6_q1(int MR);
SweepV6Launch sweep_v6_q2(int MR);
SweepV6Launch sweep_v6_q3(int MR);
SweepV6Launch sweep_v6_q4(int MR);

// Arguments of the CTA-cooperative sweep (sweep3_impl.cuh), launched with kV3Threads threads.
constexpr int kV3Threads = 512;
struct SweepV3Args {
  const float2* y;
  const int* shift;
  int N, Kp1, M, L, Lw;
  int ns;          // ring stages
  int slot_bytes;  // bytes per ring slot (an odd number of 16-byte words)
  int cp, sp, dp;  // per-image pitches (odd) of the c/W, s/w and unit-weight buffers
  int nd;          // distance units in the table: L/2 + 1 for the whole circle, else Lw
  int wrap;        // 1: the window is the whole circle (Lw == L), indices wrap
  int r0, d1;      // first reference (window index) and the distance pass 1 covers
  int fsplit;      // threads per forward item (1 or 2)
  int phase0;      // (l0 + r0) mod L on the grid; 0 for a dense window (the reference's
                   // rotation is then the window twiddle tw[k][r0])
  int off_ring, off_x, off_xr, off_td, off_tf, off_lr, off_c, off_s, off_w2, off_info, off_wl;
  float two_beta;
  double two_beta_d;
  const float2* x32;
  const float2* td;  // [Kp1][nd] (cos t - 1, -sin t), t = 2 pi k d step / L
  const float2* tf32;
  const float2* tw;  // dense window only (else null): [Kp1][twp] e^{-i k theta_{l0+i}}
  int twp;
  const float* logrho32;
  double* part;
  float* w_out;
  Ctrl* ctrl;
};
typedef void (*SweepV3Fn)(const SweepV3Args);
// QH = float4 per row (Q / 2); bi = images per batch (16, 12, 8 or 4); yf = 1 for y
// stored as the BF16 hi/lo split.
SweepV3Fn sweep_v3_qh4(int bi, int yf);
SweepV3Fn sweep_v3_qh8(int bi, int yf);
SweepV3Fn sweep_v3_qh12(int bi, int yf);
SweepV3Fn sweep_v3_qh16(int bi, int yf);

// Arguments of the chunked two-read sweep (sweep4_impl.cuh).
struct SweepV4Args {
  const float2* y;
  const int* shift;
  int N, Kp1, M, L, Lw;
  int slot_bytes;  // bytes per warp slot
  int cp, sp, dp;  // per-image pitches of the c/W, s/w and unit-weight buffers
  int nd, wrap, r0, d1, phase0;  // as in SweepV3Args
  int lc;          // log2 of the images per chunk
  int off_ring, off_x, off_td, off_tf, off_lr, off_c, off_s, off_w2, off_info, off_wl;
  float two_beta;
  const float2* x32;
  const float2* td;
  const float2* tf32;
  const float2* tw;  // as in SweepV3Args
  int twp;
  const float* logrho32;
  double* part;
  float* w_out;
  Ctrl* ctrl;
};
struct SweepV4Launch {
  void (*fn)(const SweepV4Args);
  int threads;
  int ctas_per_sm;
};
// QV = float4 per lane per row (Q / 8); MR = rows per quad ((K+1+7)/8, at most 7);
// cpsm = resident CTAs per SM (1: 512 threads, 2: 256 threads each; 256 threads and one
// CTA per SM for the largest per-lane accumulators).
// yf: 1 for y stored as the BF16 hi/lo split (load_y4), one translation unit per (QV, yf).
SweepV4Launch sweep_v4_q1_f0(int MR, int cpsm);
SweepV4Launch sweep_v4_q2_f0(int MR, int cpsm);
SweepV4Launch sweep_v4_q3_f0(int MR, int cpsm);
SweepV4Launch sweep_v4_q4_f0(int MR, int cpsm);
SweepV4Launch sweep_v4_q1_f1(int MR, int cpsm);
SweepV4Launch sweep_v4_q2_f1(int MR, int cpsm);
SweepV4Launch sweep_v4_q3_f1(int MR, int cpsm);
SweepV4Launch sweep_v4_q4_f1(int MR, int cpsm);

// Arguments of the split sweep (sweep_tc_impl.cuh): correlation, tensor-core transform and
// accumulation kernels launched in turn.
struct SplitArgs {
  const float2* y;
  const int* shift;
  int N, Kp1, M, L, Lw;
  int nwarps, slot_bytes;           // stream kernels: active warps per CTA, bytes per ring slot
  int off_ring, off_x, off_tf;
  int NP, ncols;                    // transform: window columns padded to 16, tensor-memory columns
  int k2_off_b, k2_off_ah, k2_off_al, k2_off_lr, k2_off_tf, k2_off_wt, k2_off_ll;
  int k2_off_cs;                    // transform: the tile's c (then W) rows [128][Kp1] float2, at the end the CTA's ll sums
  int k2_off_td;                    // transform: the distance-unit table's first k2_ndp distances, or 0
  int k2_ndp;                       // distances of the table in shared memory (the rest read from global)
  int k2_off_info;                  // transform: per-image peaks, distances, scales and bounds
  int wrap, l0m, nd, twp;
  float two_beta;
  const float2* x32;
  const float2* tf32;
  const float2* td;                 // [Kp1][nd] (cos t - 1, -sin t)
  const float2* tw;                 // dense window only (else null): [Kp1][twp] e^{-i k theta_l}
  const float* logrho32;
  const void* tcb;                  // [NP][KA] FP16 operand layout: (cos, sin) of k theta_l, KA = 2 KP to 16
  float2* cbuf;                     // [N][Kp1] aligned correlations
  float2* wbuf;                     // [N][Kp1] back-transformed weights W_jk
  double* part;
  int G;
  float* w_out;
  Ctrl* ctrl;
};
constexpr int kTcTile = 128;            // split sweep: images per transform tile (the MMA's M)
constexpr int kTcStreamThreads = 512;   // split sweep: threads of the streaming kernels
constexpr int kTcTransThreads = 512;    // split sweep: threads of the transform kernel
struct SplitStreamFns {
  void (*corr)(const SplitArgs);
  void (*accum)(const SplitArgs);
};
SplitStreamFns sweep_tc_q1(int MR);
SplitStreamFns sweep_tc_q2(int MR);
SplitStreamFns sweep_tc_q3(int MR);
SplitStreamFns sweep_tc_q4(int MR);
typedef void (*SplitTransFn)(const SplitArgs);
SplitTransFn sweep_tc_trans(int KP);  // KP = K+1 rounded up to 4, at most 48

// Mirror units of a window: offsets o and -o (mod L) share cos/sin.  Writes the
// (a, b) index pairs in window order of a; returns the number of units.  A dense window
// (angles step != 1 grid units apart) pairs positions l0 + i and -(l0 + i) without the
// modular wrap, which holds only on the grid.
__host__ __device__ inline int window_units(int L, int Lw, int l0, bool dense, int2* out) {
  int nu = 0;
  for (int i = 0; i < Lw; ++i) {
    int im;
    if (dense) {
      im = -2 * l0 - i;
      if (im < 0) im = Lw;  // no mirror
    } else {
      int off = (l0 + i) % L;
      if (off < 0) off += L;
      const int moff = (L - off) % L;
      im = (moff - l0) % L;
      if (im < 0) im += L;
    }
    if (im < Lw && im != i) {
      if (im < i) continue;  // covered by the unit of its mirror
      if (out) out[nu] = make_int2(i, im);
    } else {
      if (out) out[nu] = make_int2(i, -1);
    }
    ++nu;
  }
  return nu;
}
// A window of Lw rotations 2 pi step (l0 + i) / L: on the grid (step 1) 1 <= Lw <= L; a dense
// window has 0 < step < 1 and spans less than the circle, (Lw - 1) step < L, so that no two of
// its rotations coincide.
inline bool window_ok(int L, int Lw, int l0, double step) {
  if (L < 1 || Lw < 1 || l0 < -(1 << 30) || l0 > (1 << 30)) return false;
  if (step == 1.0) return Lw <= L;
  if (!(step > 0.0 && step < 1.0)) return false;
  if (Lw > (1 << 16) || l0 < -(1 << 24) || l0 > (1 << 24)) return false;
  return (double)(Lw - 1) * step < (double)L;
}

// Device properties cached per device.
struct DevInfo {
  int sms;
  int max_smem_optin;  // per CTA
  int smem_per_sm;     // shared memory of one SM (shared by its resident CTAs)
};
constexpr int kMaxCtasPerSm = 2;  // the EM partial-sum layout has room for this many CTAs per SM
int dev_info(DevInfo* out);
// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it).
int raise_smem_limit(const void* fn, int bytes);
int sweep_grid();  // persistent grid used by the sweep on the current device

}  // namespace mra
