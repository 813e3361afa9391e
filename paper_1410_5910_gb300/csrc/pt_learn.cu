// Learned correction of the preconditioner (not in the paper): a 4-layer
// network N_theta on interface traces, used in flexible GMRES (Section 4.2)
// as z = K^{-1} v + N_theta(v), with K^{-1} the Gauss-Seidel sweeps of
// Algorithm 4.  These are its training and inference kernels.
//
// Network (one sequence of n_t positions per interface and source, 8 real
// channels = Re/Im of the interface's four rows of the permuted residual):
//   h1 = b1 + W1 * x          (cross-correlation over x, kernel 7, zero padded)
//   h2 = b2 + W2 g(h1), h3 = b3 + W3 g(h2), y = b4 + W4 g(h3)   (pointwise)
// with g the tanh form of GELU.  Weights are stored in BF16 for the products
// (FP32 master copy for training), activations and accumulation in FP32.
// Activations are channel-major: act[c * P + pos], pos = seq * n_t + x.
//
// Every product is one tiled FP32 GEMM kernel (64 x 64 tile, 16-deep k
// slices in shared memory, 4 x 4 outputs per thread) with operand modes for
// transposed weights, the convolution gather (k = c * 7 + j reads
// x[c][pos + j - 3] inside the sequence) and its transpose, and epilogues for
// bias + GELU and for split-k accumulation of weight gradients.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "pt_common.cuh"

namespace pt {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kGT = 64;   // output tile
constexpr int kGK = 16;   // k slice

enum BMode { kBRow = 0, kBTrans = 1, kBConv = 2, kBConvT = 3 };
enum Epi { kEpiStore = 0, kEpiGelu = 1, kEpiGeluOnly = 2, kEpiAtomic = 3 };

struct GemmArgs {
  int M, N, K;
  const void* A;
  int lda;          // A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]
  const float* B;
  long ldb;         // kBRow: B[k * ldb + n]; kBTrans: B[n * ldb + k]; conv: channel stride
  float* C;
  long ldc;         // C[m * ldc + n]
  float* C2;        // kEpiGelu: activation output, same layout as C
  const float* bias;
  int nt;           // positions per sequence (convolution modes)
  int kchunk;       // k range of one blockIdx.z (split k)
};

__device__ __forceinline__ float gelu_f(float x) {
  const float c = 0.7978845608028654f;  // sqrt(2 / pi)
  return 0.5f * x * (1.f + tanhf(c * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float c = 0.7978845608028654f;
  const float th = tanhf(c * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * c * (1.f + 3.f * 0.044715f * x * x);
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// x[c][pos + j - half] inside pos's sequence, else 0
__device__ __forceinline__ float conv_tap(const GemmArgs& g, int c, int j, long pos) {
  const int x = (int)(pos % g.nt) + j - kNnK1 / 2;
  if (x < 0 || x >= g.nt) return 0.f;
  return g.B[(long)c * g.ldb + pos + j - kNnK1 / 2];
}

template <int TA, int BM, int EPI, typename TAe>
__global__ void __launch_bounds__(256) nn_gemm_kernel(GemmArgs g) {
  __shared__ float As[kGK][kGT + 4];
  __shared__ float Bs[kGK][kGT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long n0 = (long)blockIdx.x * kGT;
  const int m0 = blockIdx.y * kGT;
  const long kbeg = (long)blockIdx.z * g.kchunk;
  const long kend = min((long)g.K, kbeg + g.kchunk);
  const TAe* A = static_cast<const TAe*>(g.A);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (long k0 = kbeg; k0 < kend; k0 += kGK) {
    for (int q = tid; q < kGT * kGK; q += 256) {
      int mm, kk;
      if (TA) { mm = q % kGT; kk = q / kGT; } else { kk = q % kGK; mm = q / kGK; }
      const int m = m0 + mm;
      const long k = k0 + kk;
      float v = 0.f;
      if (m < g.M && k < kend) v = to_f<TAe>(TA ? A[k * g.lda + m] : A[(long)m * g.lda + k]);
      As[kk][mm] = v;
    }
    for (int q = tid; q < kGT * kGK; q += 256) {
      int kk, nn;
      if (BM == kBTrans || BM == kBConvT) { kk = q % kGK; nn = q / kGK; } else { nn = q % kGT; kk = q / kGT; }
      const long k = k0 + kk, n = n0 + nn;
      float v = 0.f;
      if (k < kend && n < g.N) {
        if (BM == kBRow) v = g.B[k * g.ldb + n];
        else if (BM == kBTrans) v = g.B[n * g.ldb + k];
        else if (BM == kBConv) v = conv_tap(g, (int)(k / kNnK1), (int)(k % kNnK1), n);
        else v = conv_tap(g, (int)(n / kNnK1), (int)(n % kNnK1), k);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      float* dst = g.C + (long)m * g.ldc + n;
      if (EPI == kEpiAtomic) {
        atomicAdd(dst, v);
      } else {
        if (g.bias) v += g.bias[m];
        if (EPI == kEpiGeluOnly) {
          *dst = gelu_f(v);
        } else {
          *dst = v;
          if (EPI == kEpiGelu) g.C2[(long)m * g.ldc + n] = gelu_f(v);
        }
      }
    }
  }
}

template <int TA, int BM, int EPI, typename TAe>
cudaError_t gemm(const GemmArgs& a, int splits, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + kGT - 1) / kGT), (unsigned)((a.M + kGT - 1) / kGT), (unsigned)splits);
  nn_gemm_kernel<TA, BM, EPI, TAe><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

GemmArgs args(int M, long N, long K, const void* A, int lda, const float* B, long ldb, float* C, long ldc) {
  GemmArgs g{};
  g.M = M;
  g.N = (int)N;
  g.K = (int)K;
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.kchunk = (int)K;
  return g;
}

__global__ void gelu_back_kernel(const float* __restrict__ dA, const float* __restrict__ H, float* __restrict__ dH,
                                 long n) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    dH[q] = dA[q] * gelu_grad_f(H[q]);
}

// dY = (Y - T) / n, loss += 0.5 * sum (Y - T)^2 / n
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY, long n,
                            double* __restrict__ loss) {
  double acc = 0.0;
  const float inv = 1.0f / (float)n;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const float d = Y[q] - T[q];
    dY[q] = d * inv;
    acc += (double)d * d;
  }
  acc = warp_sum(acc);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(loss, 0.5 * v / (double)n);
  }
}

// db[m] += sum_pos dH[m][pos]
__global__ void rowsum_kernel(const float* __restrict__ dH, long P, float* __restrict__ db) {
  const int m = blockIdx.x;
  double acc = 0.0;
  for (long q = threadIdx.x; q < P; q += blockDim.x) acc += dH[(long)m * P + q];
  acc = warp_sum(acc);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) db[m] += (float)v;
  }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, __nv_bfloat16* __restrict__ wbf, long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const float g = grad[q];
    const float mq = b1 * m[q] + (1.f - b1) * g;
    const float vq = b2 * v[q] + (1.f - b2) * g * g;
    m[q] = mq;
    v[q] = vq;
    const float t = theta[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    theta[q] = t;
    wbf[q] = __float2bfloat16(t);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf, long n) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    wbf[q] = __float2bfloat16(theta[q]);
}

// per-source RMS of a trace vector (N complex entries); zero for a zero vector
__global__ void rms_kernel(const cd* __restrict__ v, size_t N, double* __restrict__ rms) {
  const int s = blockIdx.x;
  double acc = 0.0;
  for (size_t q = threadIdx.x; q < N; q += blockDim.x) {
    const cd a = v[(size_t)s * N + q];
    acc += a.x * a.x + a.y * a.y;
  }
  acc = warp_sum(acc);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    x = warp_sum(x);
    if (threadIdx.x == 0) rms[s] = sqrt(x / (double)N);
  }
}

// features: X[ch * ldx + pos] = channel ch of v / rms for pos = ((s - s0) (L - 1) + i) n_t + x
__global__ void feat_kernel(const cd* __restrict__ v, int s0, int ns, int L, int nt, const double* __restrict__ rms,
                            float* __restrict__ X, long ldx) {
  const int T = 2 * (L - 1);
  const long P = (long)ns * (L - 1) * nt;
  for (long pos = blockIdx.x * (long)blockDim.x + threadIdx.x; pos < P; pos += (long)gridDim.x * blockDim.x) {
    const int x = (int)(pos % nt);
    const long seq = pos / nt;
    const int i = (int)(seq % (L - 1));
    const int s = s0 + (int)(seq / (L - 1));
    const double r = rms[s];
    const double inv = r > 0.0 ? 1.0 / r : 0.0;
    const cd* vs = v + (size_t)s * 2 * T * nt;
    const int tr[4] = {2 * i, 2 * i + 1, T + 2 * i, T + 2 * i + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const cd a = vs[(size_t)tr[q] * nt + x];
      X[(long)(2 * q) * ldx + pos] = (float)(a.x * inv);
      X[(long)(2 * q + 1) * ldx + pos] = (float)(a.y * inv);
    }
  }
}

// z[s] (+)= rms_s * unfeatures(Y)
__global__ void unfeat_kernel(const float* __restrict__ Y, int s0, int ns, int L, int nt,
                              const double* __restrict__ rms, cd* __restrict__ z, int add) {
  const int T = 2 * (L - 1);
  const long P = (long)ns * (L - 1) * nt;
  for (long pos = blockIdx.x * (long)blockDim.x + threadIdx.x; pos < P; pos += (long)gridDim.x * blockDim.x) {
    const int x = (int)(pos % nt);
    const long seq = pos / nt;
    const int i = (int)(seq % (L - 1));
    const int s = s0 + (int)(seq / (L - 1));
    const double r = rms[s];
    cd* zs = z + (size_t)s * 2 * T * nt;
    const int tr[4] = {2 * i, 2 * i + 1, T + 2 * i, T + 2 * i + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float yr = Y[(long)(2 * q) * P + pos], yi = Y[(long)(2 * q + 1) * P + pos];
      // a non-finite network output contributes nothing (the plain preconditioner stands)
      const bool ok = isfinite(yr) && isfinite(yi);
      const cd c = ok ? make_double2(r * (double)yr, r * (double)yi) : make_double2(0.0, 0.0);
      cd* dst = zs + (size_t)tr[q] * nt + x;
      *dst = add ? cadd(*dst, c) : c;
    }
  }
}

// gather the feature columns of a batch of pairs: dst[ch][(b (L-1) + i) n_t + x] = src[ch][(idx[b] (L-1) + i) n_t + x]
__global__ void gather_kernel(const float* __restrict__ src, long Psrc, const int* __restrict__ idx, int nb,
                              int seq_per, int nt, float* __restrict__ dst) {
  const long per = (long)seq_per * nt;
  const long P = (long)nb * per;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < (long)kNnCin * P;
       q += (long)gridDim.x * blockDim.x) {
    const int ch = (int)(q / P);
    const long pos = q % P;
    const int b = (int)(pos / per);
    const long off = pos % per;
    dst[q] = src[(long)ch * Psrc + (long)idx[b] * per + off];
  }
}

// t = e - k (complex trace vectors, n entries)
__global__ void sub_cd_kernel(const cd* __restrict__ e, const cd* __restrict__ k, cd* __restrict__ t, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    t[q] = csub(e[q], k[q]);
}

__global__ void sumsq_kernel(const float* __restrict__ x, long n, double* __restrict__ out) {
  double acc = 0.0;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    acc += (double)x[q] * x[q];
  acc = warp_sum(acc);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}

__global__ void scale_kernel(float* __restrict__ x, long n, float a) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) x[q] *= a;
}

int grid_for(long n) { return (int)std::min<long>(4 * 152 * 4, (n + 255) / 256); }

}  // namespace

// ---- host entry points used by the C ABI ----------------------------------------

static int splits_for(long P) {
  const long s = (P + 4095) / 4096;
  return (int)std::max<long>(1, std::min<long>(s, 256));
}
static int kchunk_for(long P, int splits) { return (int)(((P + splits - 1) / splits + kGK - 1) / kGK * kGK); }

// Forward pass on features X (8 x P).  w: BF16 weights, theta: FP32 master
// copy (biases are read from it).  With H non-null the pre-activations
// H1 | H2 | H3 (each W x P) are kept and A holds A1 | A2 | A3 (training);
// otherwise A holds two W x P ping-pong buffers (inference).
cudaError_t nn_forward(const __nv_bfloat16* w, const float* theta, const float* X, long P, int nt, float* H, float* A,
                       float* Y, cudaStream_t s) {
  const long WP = (long)kNnW * P;
  const bool keep = H != nullptr;
  float* A1 = A;
  float* A2 = A + WP;
  float* A3 = keep ? A + 2 * WP : A;
  cudaError_t e;
  {
    GemmArgs g = args(kNnW, P, (long)kNnCin * kNnK1, w + kNnOffW1, kNnCin * kNnK1, X, P, keep ? H : A1, P);
    g.bias = theta + kNnOffB1;
    g.nt = nt;
    g.C2 = A1;
    e = keep ? gemm<0, kBConv, kEpiGelu, __nv_bfloat16>(g, 1, s) : gemm<0, kBConv, kEpiGeluOnly, __nv_bfloat16>(g, 1, s);
    if (e != cudaSuccess) return e;
  }
  {
    GemmArgs g = args(kNnW, P, kNnW, w + kNnOffW2, kNnW, A1, P, keep ? H + WP : A2, P);
    g.bias = theta + kNnOffB2;
    g.C2 = A2;
    e = keep ? gemm<0, kBRow, kEpiGelu, __nv_bfloat16>(g, 1, s) : gemm<0, kBRow, kEpiGeluOnly, __nv_bfloat16>(g, 1, s);
    if (e != cudaSuccess) return e;
  }
  {
    GemmArgs g = args(kNnW, P, kNnW, w + kNnOffW3, kNnW, A2, P, keep ? H + 2 * WP : A3, P);
    g.bias = theta + kNnOffB3;
    g.C2 = A3;
    e = keep ? gemm<0, kBRow, kEpiGelu, __nv_bfloat16>(g, 1, s) : gemm<0, kBRow, kEpiGeluOnly, __nv_bfloat16>(g, 1, s);
    if (e != cudaSuccess) return e;
  }
  GemmArgs g = args(kNnCin, P, kNnW, w + kNnOffW4, kNnW, A3, P, Y, P);
  g.bias = theta + kNnOffB4;
  return gemm<0, kBRow, kEpiStore, __nv_bfloat16>(g, 1, s);
}

// Loss 0.5 mean (Y - T)^2 (added to *loss) and its gradient (added to grad, which the
// caller zeroes) after nn_forward with kept intermediates.  dY: 8 x P; dA, dH: W x P.
cudaError_t nn_backward(const __nv_bfloat16* w, const float* X, long P, int nt, const float* H, const float* A,
                        const float* Y, const float* T, float* dY, float* dA, float* dH, float* grad, double* loss,
                        cudaStream_t s) {
  const long WP = (long)kNnW * P;
  const float* H1 = H;
  const float* H2 = H + WP;
  const float* H3 = H + 2 * WP;
  const float* A1 = A;
  const float* A2 = A + WP;
  const float* A3 = A + 2 * WP;
  const int sp = splits_for(P), kc = kchunk_for(P, sp);
  cudaError_t e;
  loss_kernel<<<grid_for((long)kNnCin * P), 256, 0, s>>>(Y, T, dY, (long)kNnCin * P, loss);
  // weight gradient dW += dOut . In^T (split k over positions, atomics)
  auto wgrad = [&](int M, int N, const float* dOut, const float* In, float* dst) {
    GemmArgs g = args(M, N, P, dOut, (int)P, In, P, dst, N);
    g.kchunk = kc;
    return gemm<0, kBTrans, kEpiAtomic, float>(g, sp, s);
  };
  // input gradient dIn = W^T dOut (W: out x in, BF16)
  auto igrad = [&](int in, int out, size_t woff, const float* dOut, float* dst) {
    GemmArgs g = args(in, P, out, w + woff, in, dOut, P, dst, P);
    return gemm<1, kBRow, kEpiStore, __nv_bfloat16>(g, 1, s);
  };
  if ((e = wgrad(kNnCin, kNnW, dY, A3, grad + kNnOffW4)) != cudaSuccess) return e;
  rowsum_kernel<<<kNnCin, 256, 0, s>>>(dY, P, grad + kNnOffB4);
  if ((e = igrad(kNnW, kNnCin, kNnOffW4, dY, dA)) != cudaSuccess) return e;
  gelu_back_kernel<<<grid_for(WP), 256, 0, s>>>(dA, H3, dH, WP);
  if ((e = wgrad(kNnW, kNnW, dH, A2, grad + kNnOffW3)) != cudaSuccess) return e;
  rowsum_kernel<<<kNnW, 256, 0, s>>>(dH, P, grad + kNnOffB3);
  if ((e = igrad(kNnW, kNnW, kNnOffW3, dH, dA)) != cudaSuccess) return e;
  gelu_back_kernel<<<grid_for(WP), 256, 0, s>>>(dA, H2, dH, WP);
  if ((e = wgrad(kNnW, kNnW, dH, A1, grad + kNnOffW2)) != cudaSuccess) return e;
  rowsum_kernel<<<kNnW, 256, 0, s>>>(dH, P, grad + kNnOffB2);
  if ((e = igrad(kNnW, kNnW, kNnOffW2, dH, dA)) != cudaSuccess) return e;
  gelu_back_kernel<<<grid_for(WP), 256, 0, s>>>(dA, H1, dH, WP);
  {
    GemmArgs g = args(kNnW, (long)kNnCin * kNnK1, P, dH, (int)P, X, P, grad + kNnOffW1, (long)kNnCin * kNnK1);
    g.kchunk = kc;
    g.nt = nt;
    if ((e = gemm<0, kBConvT, kEpiAtomic, float>(g, sp, s)) != cudaSuccess) return e;
  }
  rowsum_kernel<<<kNnW, 256, 0, s>>>(dH, P, grad + kNnOffB1);
  return cudaGetLastError();
}

cudaError_t nn_to_bf16(const float* theta, __nv_bfloat16* wbf, cudaStream_t s) {
  to_bf16_kernel<<<grid_for(kNnParams), 256, 0, s>>>(theta, wbf, (long)kNnParams);
  return cudaGetLastError();
}

// Adam (Kingma & Ba): step t >= 1, moments m, v, bias corrections 1 - b^t
cudaError_t nn_adam(float* theta, float* m, float* v, const float* grad, __nv_bfloat16* wbf, double lr, int t,
                    cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, t)), c2 = (float)(1.0 - std::pow(b2, t));
  adam_kernel<<<grid_for(kNnParams), 256, 0, s>>>(theta, m, v, grad, wbf, (long)kNnParams, (float)lr, (float)b1,
                                                   (float)b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t nn_rms(const cd* v, int S, size_t N, double* rms, cudaStream_t s) {
  rms_kernel<<<S, 256, 0, s>>>(v, N, rms);
  return cudaGetLastError();
}

cudaError_t nn_features(const cd* v, int s0, int ns, int L, int nt, const double* rms, float* X, long ldx,
                        cudaStream_t s) {
  feat_kernel<<<grid_for((long)ns * (L - 1) * nt), 256, 0, s>>>(v, s0, ns, L, nt, rms, X, ldx);
  return cudaGetLastError();
}

cudaError_t nn_unfeatures(const float* Y, int s0, int ns, int L, int nt, const double* rms, cd* z, bool add,
                          cudaStream_t s) {
  unfeat_kernel<<<grid_for((long)ns * (L - 1) * nt), 256, 0, s>>>(Y, s0, ns, L, nt, rms, z, add ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t nn_gather(const float* src, long Psrc, const int* idx, int nb, int seq_per, int nt, float* dst,
                      cudaStream_t s) {
  gather_kernel<<<grid_for((long)kNnCin * nb * seq_per * nt), 256, 0, s>>>(src, Psrc, idx, nb, seq_per, nt, dst);
  return cudaGetLastError();
}

// *out += sum x^2 (caller zeroes *out)
cudaError_t nn_sumsq(const float* x, long n, double* out, cudaStream_t s) {
  sumsq_kernel<<<grid_for(n), 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t nn_scale(float* x, long n, float a, cudaStream_t s) {
  scale_kernel<<<grid_for(n), 256, 0, s>>>(x, n, a);
  return cudaGetLastError();
}

cudaError_t nn_sub(const cd* e, const cd* k, cd* t, size_t n, cudaStream_t s) {
  sub_cd_kernel<<<grid_for((long)n), 256, 0, s>>>(e, k, t, n);
  return cudaGetLastError();
}

}  // namespace pt
