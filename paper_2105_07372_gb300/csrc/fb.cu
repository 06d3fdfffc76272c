// Fourier-Bessel front end (App. A): from n x n pixel images to the steerable coefficients
// a_{k,q} (k = 0..K, q = 1..Q) as the least-squares solution over the sampled basis.
//
//   setup    (once per n, K, Q)  Bessel zeros R_{k,q} (scan and bisection of J_k, FP64), the real
//            design matrix A [n^2 x Mr] (Mr = Q + 2KQ: a_0q, then Re a_kq and Im a_kq of
//            u^{kq} + u^{-kq}), its Gram G = A^T A (cuBLAS DGEMM), G^{-1} by Newton-Schulz from
//            the Jacobi start diag(G)^{-1} (DGEMMs; the Jacobi-scaled Gram of the sampled basis is
//            within ~1% of the identity, so a few steps reach FP64 accuracy), the projection
//            P = G^{-1} A^T, stored per pixel in the coefficient layout [n^2][K+1][Q] complex FP32.
//   pack     P transposed and split into three BF16 pieces in the tiled operand layout of the
//            tcgen05 GEMM (gemm3.cuh), once per P.
//   project  y = images P, one GEMM over all images: [N x n^2] by [n^2 x 2M] on the tensor cores
//            (k_gemm3: six BF16 products of the three-piece split, FP32 accumulation; three in the
//            fast mode).
//
// Basis (App. A): u^{k,q}(r, theta) = N_{k,q} J_|k|(R_{|k|,q} r / c) e^{i k theta} on r <= c = (n - 1)/2,
// N_{k,q} = 1 / (c sqrt(pi) |J_{k+1}(R_{k,q})|); pixel (row iy, column ix) at x = ix - c, y = iy - c.
#include <cublas_v2.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"
#include "gemm3.cuh"

namespace mra {
namespace {

// q-th positive zeros of J_k for k = 0..K, one warp per k: the grid x_j = x0 + j h (h = 0.05; zeros
// are ~pi apart) from x0 = max(k, h) (the first zero of J_k lies above k) up to beyond McMahon's
// estimate of the Q-th zero, split into 32 consecutive runs of grid intervals; each lane counts the
// sign changes in its run, a warp prefix sum orders them, and each lane then bisects its own
// changes (80 halvings) into R[k][q]; also the normalisation N_{k,q}.
__global__ void k_fb_zeros(int K, int Q, double c, double* R, double* Nkq, int* status) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k > K) return;
  const double h = 0.05;
  const double x0 = k == 0 ? h : (double)k;
  const double xmax = (Q + 0.5 * k + 2.0) * M_PI + 2.0;
  const long long nint = (long long)((xmax - x0) / h) + 1;  // grid intervals scanned
  const long long per = (nint + 31) / 32;
  const long long j0 = lane * per, j1 = min(nint, j0 + per);
  auto count = [&](bool write, int base) {
    int n = 0;
    if (j0 >= j1) return 0;
    double xa = x0 + (double)j0 * h, fa = jn(k, xa);
    for (long long j = j0; j < j1; ++j) {
      const double xb = x0 + (double)(j + 1) * h, fb = jn(k, xb);
      if ((fa < 0.0) != (fb < 0.0)) {
        if (write && base + n < Q) {
          double lo = xa, hi = xb, flo = fa;
          for (int it = 0; it < 80; ++it) {
            const double mid = 0.5 * (lo + hi), fm = jn(k, mid);
            if ((fm < 0.0) == (flo < 0.0)) lo = mid, flo = fm; else hi = mid;
          }
          const double z = 0.5 * (lo + hi);
          R[k * Q + base + n] = z;
          Nkq[k * Q + base + n] = 1.0 / (c * sqrt(M_PI) * fabs(jn(k + 1, z)));
        }
        ++n;
      }
      xa = xb, fa = fb;
    }
    return n;
  };
  const int mine = count(false, 0);
  int incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total < Q) {
    if (lane == 0) atomicExch(status, (int)MRA_ENUMERIC);
    return;
  }
  if (incl - mine < Q) count(true, incl - mine);
}

// At[col][pixel] (row-major [Mr][n^2]): the design matrix column by column.
__global__ void k_fb_basis(int n, int K, int Q, double c, const double* R, const double* Nkq, double* At) {
  const long long npix = (long long)n * n, Mr = Q + 2LL * K * Q;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < Mr * npix;
       idx += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(idx / npix);
    const int pix = (int)(idx - (long long)col * npix);
    int k, q, part;
    if (col < Q) {
      k = 0, q = col, part = 0;
    } else {
      const int j = col - Q;
      k = 1 + j / (2 * Q);
      q = (j % (2 * Q)) / 2;
      part = j & 1;
    }
    const double x = (double)(pix % n) - c, y = (double)(pix / n) - c;
    const double r = sqrt(x * x + y * y);
    double v = 0.0;
    if (r <= c) {
      // J_k(0) = 1 for k = 0 and 0 otherwise (the library's jn is not evaluated at 0 for k >= 2)
      const double jk = r > 0.0 ? jn(k, R[k * Q + q] * r / c) : (k == 0 ? 1.0 : 0.0);
      const double f = Nkq[k * Q + q] * jk;
      if (k == 0) {
        v = f;
      } else {
        double s, co;
        sincos((double)k * atan2(y, x), &s, &co);
        v = part == 0 ? 2.0 * f * co : -2.0 * f * s;
      }
    }
    At[idx] = v;
  }
}

// X = diag(G)^{-1} (column-major Mr x Mr)
__global__ void k_fb_jacobi(int Mr, const double* G, double* X) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)Mr * Mr;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % Mr), j = (int)(idx / Mr);
    X[idx] = i == j ? 1.0 / G[idx] : 0.0;
  }
}

// P (column-major [Mr x n^2], i.e. per pixel the Mr real parameters) to the coefficient layout
// out[pixel][k][q] = (Re, Im) in FP32, Im = 0 for k = 0.
__global__ void k_fb_scatter(int npix, int K, int Q, const double* P, float2* out) {
  const int Mr = Q + 2 * K * Q, M = (K + 1) * Q;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)npix * M;
       idx += (long long)gridDim.x * blockDim.x) {
    const int pix = (int)(idx / M), e = (int)(idx % M);
    const int k = e / Q, q = e % Q;
    const double* p = P + (size_t)pix * Mr;
    float2 v;
    if (k == 0) {
      v = make_float2((float)p[q], 0.f);
    } else {
      const int col = Q + 2 * ((k - 1) * Q + q);
      v = make_float2((float)p[col], (float)p[col + 1]);
    }
    out[idx] = v;
  }
}

// status = MRA_ENUMERIC if max |T - I| > tol (T column-major Mr x Mr): the iteration did not reach G^{-1}.
__global__ void k_fb_check(int Mr, const double* T, double tol, int* status) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)Mr * Mr;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % Mr), j = (int)(idx / Mr);
    const double e = T[idx] - (i == j ? 1.0 : 0.0);
    if (!(fabs(e) <= tol)) atomicExch(status, (int)MRA_ENUMERIC);
  }
}

// One cuBLAS handle per device, created on first use.
int blas_handle(cublasHandle_t* out) {
  static std::mutex mu;
  static std::map<int, cublasHandle_t> handles;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MRA_ECUDA;
  std::lock_guard<std::mutex> g(mu);
  auto it = handles.find(dev);
  if (it == handles.end()) {
    cublasHandle_t h;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return MRA_ECUDA;
    it = handles.emplace(dev, h).first;
  }
  *out = it->second;
  return MRA_OK;
}

struct FbLayout {
  size_t R, N, status, At, G, X, T, Xn, P, total;
};
FbLayout fb_layout(int n, int K, int Q) {
  const size_t npix = (size_t)n * n, Mr = (size_t)Q + 2 * (size_t)K * Q, zq = (size_t)(K + 1) * Q;
  FbLayout l;
  size_t o = 0;
  l.R = o; o = align256(o + 8 * zq);
  l.N = o; o = align256(o + 8 * zq);
  l.status = o; o = align256(o + 16);
  l.At = o; o = align256(o + 8 * Mr * npix);
  l.G = o; o = align256(o + 8 * Mr * Mr);
  l.X = o; o = align256(o + 8 * Mr * Mr);
  l.T = o; o = align256(o + 8 * Mr * Mr);
  l.Xn = o; o = align256(o + 8 * Mr * Mr);
  l.P = o; o = align256(o + 8 * Mr * npix);
  l.total = o;
  return l;
}

bool fb_dims_ok(int n, int K, int Q) {
  if (n < 3 || n > 1024 || K < 0 || Q < 1 || K > 256 || Q > 256) return false;
  if (((K + 1) * Q) % 2 != 0) return false;
  // sampling criterion R_{k,q} <= pi n / 2 (App. A), with McMahon's estimate R_{K,Q} ~ (Q + K/2 - 1/4) pi
  // plus a margin of half a zero spacing
  return (double)Q + 0.5 * K + 0.25 <= 0.5 * n;
}

constexpr int kFbNewtonSteps = 6;  // error ~ delta^(2^6) from a Jacobi start within delta < 0.1

}  // namespace
}  // namespace mra

using namespace mra;

extern "C" {

MRA_API size_t mra_fb_setup_workspace_bytes(int32_t n, int32_t K, int32_t Q) {
  if (!fb_dims_ok(n, K, Q)) return 0;
  return fb_layout(n, K, Q).total;
}

MRA_API int mra_fb_setup(int32_t n, int32_t K, int32_t Q, float* P_out, double* zeros_out, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!fb_dims_ok(n, K, Q)) return MRA_EINVAL;
  if (!P_out || (reinterpret_cast<uintptr_t>(P_out) % 16) != 0 || !ws || (reinterpret_cast<uintptr_t>(ws) % 256) != 0)
    return MRA_EINVAL;
  if (zeros_out && (reinterpret_cast<uintptr_t>(zeros_out) % 8) != 0) return MRA_EINVAL;
  const FbLayout L_ = fb_layout(n, K, Q);
  if (ws_bytes < L_.total) return MRA_EWORKSPACE;
  cublasHandle_t h;
  if (blas_handle(&h) != MRA_OK) return MRA_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return MRA_ECUDA;
  unsigned char* b = static_cast<unsigned char*>(ws);
  double* R = reinterpret_cast<double*>(b + L_.R);
  double* Nkq = reinterpret_cast<double*>(b + L_.N);
  int* status = reinterpret_cast<int*>(b + L_.status);
  double* At = reinterpret_cast<double*>(b + L_.At);
  double* G = reinterpret_cast<double*>(b + L_.G);
  double* X = reinterpret_cast<double*>(b + L_.X);
  double* T = reinterpret_cast<double*>(b + L_.T);
  double* Xn = reinterpret_cast<double*>(b + L_.Xn);
  double* P = reinterpret_cast<double*>(b + L_.P);
  const int npix = n * n, Mr = Q + 2 * K * Q;
  const double c = 0.5 * (n - 1);
  if (cudaMemsetAsync(status, 0, 16, s) != cudaSuccess) return MRA_ECUDA;
  k_fb_zeros<<<(K + 1 + 3) / 4, 128, 0, s>>>(K, Q, c, R, Nkq, status);  // a warp per k
  k_fb_basis<<<2048, 256, 0, s>>>(n, K, Q, c, R, Nkq, At);
  if (cudaGetLastError() != cudaSuccess) return MRA_ECUDA;
  // A is column-major [npix x Mr] (At row-major); G = A^T A
  const double one = 1.0, zero = 0.0, two = 2.0, mone = -1.0;
  if (cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, Mr, Mr, npix, &one, At, npix, At, npix, &zero, G, Mr) !=
      CUBLAS_STATUS_SUCCESS)
    return MRA_ECUDA;
  k_fb_jacobi<<<1024, 256, 0, s>>>(Mr, G, X);
  for (int it = 0; it < kFbNewtonSteps; ++it) {  // X <- 2X - X G X
    if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, Mr, Mr, Mr, &one, G, Mr, X, Mr, &zero, T, Mr) !=
        CUBLAS_STATUS_SUCCESS)
      return MRA_ECUDA;
    if (cudaMemcpyAsync(Xn, X, sizeof(double) * Mr * Mr, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return MRA_ECUDA;
    if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, Mr, Mr, Mr, &mone, X, Mr, T, Mr, &two, Xn, Mr) !=
        CUBLAS_STATUS_SUCCESS)
      return MRA_ECUDA;
    std::swap(X, Xn);
  }
  // G X must be the identity to FP64 accuracy (the sampled basis is far from singular for n, K, Q
  // within the sampling criterion; otherwise the setup reports MRA_ENUMERIC)
  if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, Mr, Mr, Mr, &one, G, Mr, X, Mr, &zero, T, Mr) != CUBLAS_STATUS_SUCCESS)
    return MRA_ECUDA;
  k_fb_check<<<1024, 256, 0, s>>>(Mr, T, 1e-10, status);
  // P = X A^T, column-major [Mr x npix]
  if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, Mr, npix, Mr, &one, X, Mr, At, npix, &zero, P, Mr) !=
      CUBLAS_STATUS_SUCCESS)
    return MRA_ECUDA;
  k_fb_scatter<<<2048, 256, 0, s>>>(npix, K, Q, P, reinterpret_cast<float2*>(P_out));
  if (zeros_out &&
      cudaMemcpyAsync(zeros_out, R, sizeof(double) * (K + 1) * Q, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return MRA_ECUDA;
  if (cudaGetLastError() != cudaSuccess) return MRA_ECUDA;
  int st = 0;
  if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MRA_ECUDA;
  return st;
}

// The packed projection operand: a 256-byte header (the status word of the projection's bounded
// waits) and the tiles of P^T.
static size_t fb_operand_bytes(int n, int K, int Q) {
  const int npix = n * n, two_m = 2 * (K + 1) * Q;
  const size_t NT = (size_t)(two_m + kG3Cols - 1) / kG3Cols, KB = (size_t)(npix + kG3KB - 1) / kG3KB;
  return 256 + NT * KB * 3 * kG3BTile;
}

MRA_API size_t mra_fb_operand_bytes(int32_t n, int32_t K, int32_t Q) {
  if (!fb_dims_ok(n, K, Q)) return 0;
  return fb_operand_bytes(n, K, Q);
}

MRA_API int mra_fb_pack(int32_t n, int32_t K, int32_t Q, const float* P, void* op_out, void* stream) {
  if (!fb_dims_ok(n, K, Q) || !P || !op_out || (reinterpret_cast<uintptr_t>(P) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(op_out) % 256) != 0)
    return MRA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int npix = n * n, two_m = 2 * (K + 1) * Q;
  const int NT = (two_m + kG3Cols - 1) / kG3Cols, KB = (npix + kG3KB - 1) / kG3KB;
  unsigned char* op = static_cast<unsigned char*>(op_out);
  if (cudaMemsetAsync(op, 0, 256, s) != cudaSuccess) return MRA_ECUDA;
  // B^T(j, p) = P[p][j]: column j of the coefficient layout, pixel p
  k_gemm3_pack<<<4096, 256, 0, s>>>(P, 1, two_m, two_m, npix, NT, KB, kG3Cols, op + 256);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

MRA_API int mra_fb_project(int32_t N, int32_t n, int32_t K, int32_t Q, const float* images, const void* op,
                           float* y_out, int32_t fast, void* stream) {
  if (N < 1 || !fb_dims_ok(n, K, Q)) return MRA_EINVAL;
  if (!images || !op || !y_out || (reinterpret_cast<uintptr_t>(images) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(op) % 256) != 0 || (reinterpret_cast<uintptr_t>(y_out) % 16) != 0)
    return MRA_EINVAL;
  DevInfo di;
  if (dev_info(&di) != MRA_OK) return MRA_ECUDA;
  if (raise_smem_limit(reinterpret_cast<const void*>(k_gemm3<0>), kG3Smem) != MRA_OK) return MRA_ECUDA;
  const int npix = n * n, two_m = 2 * (K + 1) * Q;
  Gemm3Args g{};
  g.A = images;
  g.lda = npix;
  g.rows = N;
  g.K = npix;
  g.Bp = static_cast<const unsigned char*>(op) + 256;
  g.NT = (two_m + kG3Cols - 1) / kG3Cols;
  g.KB = (npix + kG3KB - 1) / kG3KB;
  g.cols = two_m;
  g.nprod = fast ? 3 : 6;
  g.brows = kG3Cols;
  g.C = y_out;
  g.ldc = two_m;
  g.status = reinterpret_cast<int*>(const_cast<void*>(op));
  const int items = ((N + kG3Rows - 1) / kG3Rows) * g.NT;
  k_gemm3<0><<<std::min(items, di.sms), kG3Threads, kG3Smem, static_cast<cudaStream_t>(stream)>>>(g);
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

}  // extern "C"

// ============================================================================ steerable PCA
// For every angular index k: the uncentred second moment C_k = (1/N) sum_i a_ik a_ik^H over the Q
// radial entries (k_spca_moments: FP64 partial sums per chunk of images), its eigen-decomposition on
// the host (C++, FP64: cyclic Jacobi on the real symmetric embedding [[Re C, -Im C], [Im C, Re C]],
// whose eigenvectors (x; y) are the complex eigenvectors x + i y, each twice; a complex Gram-Schmidt
// pass keeps one of each pair), the eigenvectors whose eigenvalue exceeds the noise-only edge
// sigma^2 (1 + sqrt(Q/N))^2, and the projection b_ik = U_k^H a_ik (k_spca_project).
#include <complex>
#include <vector>

namespace mra {
namespace {

typedef std::complex<double> cd;

// Eigen-decomposition of a Hermitian n x n matrix A (column-major): w descending, V's columns the
// eigenvectors, each scaled so that its largest-magnitude entry is real positive.
int herm_eig(int n, const cd* A, double* w, cd* V) {
  const int m = 2 * n;
  std::vector<double> S((size_t)m * m), E((size_t)m * m, 0.0);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const cd a = A[(size_t)j * n + i];  // row i, column j
      S[(size_t)j * m + i] = a.real();
      S[(size_t)(j + n) * m + i] = -a.imag();
      S[(size_t)j * m + i + n] = a.imag();
      S[(size_t)(j + n) * m + i + n] = a.real();
    }
  for (int i = 0; i < m; ++i) E[(size_t)i * m + i] = 1.0;
  auto s_at = [&](int i, int j) -> double& { return S[(size_t)j * m + i]; };
  double norm = 0.0;
  for (double v : S) norm += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < j; ++i) off += s_at(i, j) * s_at(i, j);
    if (off <= 1e-26 * norm) break;  // off-diagonal part below 1e-13 of the matrix (rounding level after that)
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = s_at(p, q);
        if (apq == 0.0) continue;
        const double theta = (s_at(q, q) - s_at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double skp = s_at(k, p), skq = s_at(k, q);
          s_at(k, p) = c * skp - s * skq;
          s_at(k, q) = s * skp + c * skq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double spk = s_at(p, k), sqk = s_at(q, k);
          s_at(p, k) = c * spk - s * sqk;
          s_at(q, k) = s * spk + c * sqk;
        }
        for (int k = 0; k < m; ++k) {
          const double ekp = E[(size_t)p * m + k], ekq = E[(size_t)q * m + k];
          E[(size_t)p * m + k] = c * ekp - s * ekq;
          E[(size_t)q * m + k] = s * ekp + c * ekq;
        }
      }
  }
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return s_at(x, x) > s_at(y, y); });
  std::vector<cd> U;  // accepted complex eigenvectors, n each
  std::vector<double> lam;
  for (int idx = 0; idx < m && (int)lam.size() < n; ++idx) {
    const int j = order[idx];
    std::vector<cd> u(n);
    for (int i = 0; i < n; ++i) u[i] = cd(E[(size_t)j * m + i], E[(size_t)j * m + i + n]);
    for (size_t v = 0; v < lam.size(); ++v) {
      cd dot = 0.0;
      for (int i = 0; i < n; ++i) dot += std::conj(U[v * n + i]) * u[i];
      for (int i = 0; i < n; ++i) u[i] -= dot * U[v * n + i];
    }
    double r = 0.0;
    for (int i = 0; i < n; ++i) r += std::norm(u[i]);
    r = std::sqrt(r);
    if (r < 0.5) continue;  // the partner of an accepted vector
    for (int i = 0; i < n; ++i) u[i] /= r;
    double l = 0.0;  // Rayleigh quotient u^H A u
    for (int jj = 0; jj < n; ++jj) {
      cd au = 0.0;
      for (int i = 0; i < n; ++i) au += A[(size_t)i * n + jj] * u[i];  // (A u)_jj = sum_i A[jj][i] u_i
      l += (std::conj(u[jj]) * au).real();
    }
    U.insert(U.end(), u.begin(), u.end());
    lam.push_back(l);
  }
  if ((int)lam.size() < n) return MRA_ENUMERIC;
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[x] > lam[y]; });
  for (int c = 0; c < n; ++c) {
    const cd* u = &U[(size_t)ord[c] * n];
    int imax = 0;
    for (int i = 1; i < n; ++i)
      if (std::abs(u[i]) > std::abs(u[imax])) imax = i;
    const cd ph = std::conj(u[imax]) / std::abs(u[imax]);
    for (int i = 0; i < n; ++i) V[(size_t)c * n + i] = u[i] * ph;
    w[c] = lam[ord[c]];
  }
  return MRA_OK;
}

// Second moments of steerable PCA: block (chunk, k) sums a_ik[q] conj(a_ik[q']) over its images into
// the FP64 partial part[k][chunk][q][q'] (each thread owns entries q Q + q' = tid, tid + 256, ...;
// images staged 64 at a time in shared memory).  k_spca_moments_sum adds the partials in chunk order.
constexpr int kSpcaChunk = 2048, kSpcaStage = 64;
__global__ void k_spca_moments(const float2* y, int N, int Kp1, int Q, int nchunk, int stage, double2* part) {
  extern __shared__ float2 sa[];  // [stage][Q]
  const int k = blockIdx.y, chunk = blockIdx.x, M = Kp1 * Q, QQ = Q * Q;
  const int i0 = chunk * kSpcaChunk, i1 = min(N, i0 + kSpcaChunk);
  double2* out = part + ((size_t)k * nchunk + chunk) * QQ;
  for (int e = threadIdx.x; e < QQ; e += blockDim.x) out[e] = make_double2(0.0, 0.0);
  for (int b = i0; b < i1; b += stage) {
    const int nb = min(stage, i1 - b);
    __syncthreads();
    for (int t = threadIdx.x; t < nb * Q; t += blockDim.x) {
      const int ii = t / Q, q = t - ii * Q;
      sa[ii * Q + q] = y[(size_t)(b + ii) * M + (size_t)k * Q + q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < QQ; e += blockDim.x) {
      const int q = e / Q, q2 = e - q * Q;
      float re = 0.f, im = 0.f;
      for (int ii = 0; ii < nb; ++ii) {
        const float2 u = sa[ii * Q + q], v = sa[ii * Q + q2];  // u conj(v)
        re = fmaf(u.x, v.x, fmaf(u.y, v.y, re));
        im = fmaf(u.y, v.x, fmaf(-u.x, v.y, im));
      }
      out[e].x += (double)re;
      out[e].y += (double)im;
    }
  }
}
__global__ void k_spca_moments_sum(const double2* part, int Kp1, int Q, int nchunk, double invN, float2* D) {
  const int QQ = Q * Q;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Kp1 * QQ; idx += gridDim.x * blockDim.x) {
    const int k = idx / QQ, e = idx - k * QQ;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const double2 v = part[((size_t)k * nchunk + c) * QQ + e];
      re += v.x, im += v.y;
    }
    // column-major Q x Q per k (entry (q, q') at q' Q + q), as the eigensolver reads it
    const int q = e / Q, q2 = e - q * Q;
    D[(size_t)k * QQ + (size_t)q2 * Q + q] = make_float2((float)(re * invN), (float)(im * invN));
  }
}

// Reduced coefficients b_ik[c] = sum_q conj(U_k[q][c]) a_ik[q] (U column-major per k), zero for c >= qc.
__global__ void k_spca_project(const float2* y, int N, int Kp1, int Q, int K2, int Q2, int qc, const float2* U,
                               float2* out) {
  const int M2 = (K2 + 1) * Q2, M = Kp1 * Q;
  const long long n = (long long)N * M2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / M2), r = (int)(idx - (long long)i * M2), k = r / Q2, c = r - k * Q2;
    float2 acc = make_float2(0.f, 0.f);
    if (c < qc) {
      const float2* a = y + (size_t)i * M + (size_t)k * Q;
      const float2* u = U + ((size_t)k * Q + c) * Q;
      for (int q = 0; q < Q; ++q) {
        const float2 av = a[q], uv = u[q];  // conj(u) a
        acc.x = fmaf(uv.x, av.x, fmaf(uv.y, av.y, acc.x));
        acc.y = fmaf(uv.x, av.y, fmaf(-uv.y, av.x, acc.y));
      }
    }
    out[idx] = acc;
  }
}

}  // namespace
}  // namespace mra

extern "C" {

MRA_API int mra_hermitian_eig(int32_t n, const double* A, double* w, double* V) {
  if (n < 1 || n > 512 || !A || !w || !V) return MRA_EINVAL;
  return herm_eig(n, reinterpret_cast<const cd*>(A), w, reinterpret_cast<cd*>(V));
}

MRA_API size_t mra_spca_workspace_bytes(const mra_dims* d) {
  if (!d || d->N < 1 || d->K < 0 || d->Q < 1 || d->Q > 512) return 0;
  const size_t QQ = (size_t)d->Q * d->Q, nchunk = ((size_t)d->N + kSpcaChunk - 1) / kSpcaChunk;
  return align256(sizeof(float) * 2 * (size_t)(d->K + 1) * QQ) + align256(sizeof(double) * 2 * (d->K + 1) * nchunk * QQ);
}

MRA_API int mra_spca_fit(const mra_dims* d, const float* y, float* basis_out, double* eig_out, int32_t* counts_out,
                         int32_t* K2_out, int32_t* Q2_out, void* ws, size_t ws_bytes, void* stream) {
  if (!d || d->N < 1 || d->K < 0 || d->Q < 1 || d->Q > 512 || !(d->sigma2 >= 0.0)) return MRA_EINVAL;
  if (!y || (reinterpret_cast<uintptr_t>(y) % 16) != 0 || !basis_out ||
      (reinterpret_cast<uintptr_t>(basis_out) % 8) != 0 || !ws || !K2_out || !Q2_out)
    return MRA_EINVAL;
  const int Kp1 = d->K + 1, Q = d->Q, M = Kp1 * Q, N = d->N;
  if (M % 2 != 0) return MRA_EINVAL;
  if (ws_bytes < mra_spca_workspace_bytes(d)) return MRA_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // C_k = (1/N) sum_i a_ik a_ik^H: entry (q, q') is the mean of a_q conj(a_q'); per-chunk FP64 partials
  // added in a fixed order
  const int nchunk = (N + kSpcaChunk - 1) / kSpcaChunk;
  cuComplex* D = static_cast<cuComplex*>(ws);
  double2* part = reinterpret_cast<double2*>(static_cast<unsigned char*>(ws) +
                                             align256(sizeof(float) * 2 * (size_t)Kp1 * Q * Q));
  const int stage = std::max(1, std::min(kSpcaStage, (96 * 1024) / (Q * 8)));  // images staged per pass
  const int sm = stage * Q * 8;
  if (sm > 48 * 1024 && raise_smem_limit(reinterpret_cast<const void*>(k_spca_moments), sm) != MRA_OK)
    return MRA_ECUDA;
  k_spca_moments<<<dim3(nchunk, Kp1), 256, sm, s>>>(reinterpret_cast<const float2*>(y), N, Kp1, Q, nchunk, stage,
                                                    part);
  k_spca_moments_sum<<<std::min(1024, (Kp1 * Q * Q + 255) / 256), 256, 0, s>>>(part, Kp1, Q, nchunk, 1.0 / N,
                                                                               reinterpret_cast<float2*>(D));
  if (cudaGetLastError() != cudaSuccess) return MRA_ECUDA;
  std::vector<cuComplex> Dh((size_t)Kp1 * Q * Q);
  if (cudaMemcpyAsync(Dh.data(), D, sizeof(cuComplex) * Dh.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MRA_ECUDA;
  const double edge = d->sigma2 * (1.0 + std::sqrt((double)Q / N)) * (1.0 + std::sqrt((double)Q / N));
  std::vector<cd> C((size_t)Q * Q), V((size_t)Q * Q);
  std::vector<double> w(Q);
  std::vector<cuComplex> Bh((size_t)Kp1 * Q * Q);
  int K2 = 0, Q2 = 1;
  for (int k = 0; k < Kp1; ++k) {
    for (size_t e = 0; e < (size_t)Q * Q; ++e) {
      const cuComplex v = Dh[(size_t)k * Q * Q + e];
      C[e] = cd(v.x, v.y);
    }
    const int st = herm_eig(Q, C.data(), w.data(), V.data());
    if (st != MRA_OK) return st;
    int keep = 0;
    while (keep < Q && w[keep] > edge) ++keep;
    if (counts_out) counts_out[k] = keep;
    if (eig_out)
      for (int q = 0; q < Q; ++q) eig_out[(size_t)k * Q + q] = w[q];
    if (keep > 0) K2 = k, Q2 = std::max(Q2, keep);
    for (int c = 0; c < Q; ++c)
      for (int i = 0; i < Q; ++i) {
        const cd v = c < keep ? V[(size_t)c * Q + i] : cd(0.0, 0.0);
        Bh[((size_t)k * Q + c) * Q + i] = make_cuComplex((float)v.real(), (float)v.imag());
      }
  }
  if (((K2 + 1) * Q2) % 2) ++Q2;
  *K2_out = K2;
  *Q2_out = Q2;
  if (cudaMemcpyAsync(basis_out, Bh.data(), sizeof(cuComplex) * Bh.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MRA_ECUDA;
  return MRA_OK;
}

MRA_API int mra_spca_project(const mra_dims* d, const float* y, int32_t K2, int32_t Q2, const float* basis,
                             float* y_out, void* stream) {
  if (!d || d->N < 1 || d->K < 0 || d->Q < 1 || d->Q > 512 || K2 < 0 || K2 > d->K || Q2 < 1 || Q2 > d->Q + 1)
    return MRA_EINVAL;
  if (!y || !basis || !y_out || (reinterpret_cast<uintptr_t>(y) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(basis) % 8) != 0 || (reinterpret_cast<uintptr_t>(y_out) % 16) != 0)
    return MRA_EINVAL;
  const int Q = d->Q, M = (d->K + 1) * Q, M2 = (K2 + 1) * Q2, N = d->N;
  if (M2 % 2 != 0) return MRA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)M;
  const int qc = std::min(Q2, Q);  // basis columns used (a padding column beyond Q stays zero)
  const long long n = (long long)N * M2;
  k_spca_project<<<(int)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const float2*>(y), N, d->K + 1, Q, K2, Q2, qc, reinterpret_cast<const float2*>(basis),
      reinterpret_cast<float2*>(y_out));
  return cudaGetLastError() == cudaSuccess ? MRA_OK : MRA_ECUDA;
}

}  // extern "C"
