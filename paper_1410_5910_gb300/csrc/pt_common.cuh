// Shared device-side definitions of the polartrace library (sm_103a).
//
// Storage conventions (see include/polartrace.h for the public layouts):
//  * local problem of layer l: z-fastest ordering inside the layer, i.e. the
//    block-tridiagonal form along x whose diagonal blocks couple the nloc
//    rows of one grid column (Section 2.2 local problem, reordered);
//  * Sinv[l][i] = (Schur complement of column i)^{-1}, nloc x nloc, row-major;
//  * W[l][i][r], E[l][i][r]: x-couplings of row r of column i to columns
//    i-1 and i+1 (diagonal off-diagonal blocks);
//  * interface blocks B[l][jk] = G^l(z_j, z_k) / h (Definition 1), n_t x n_t
//    row-major; jk = 4 * jj + kk with jj, kk in {0: j=0, 1: j=1, 2: j=n, 3: j=n+1}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <unordered_set>

namespace pt {

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum (less its
// static shared memory), once per kernel.  The limit is a per-function setting: setting
// it to each launch's own size would race between host threads that launch the same
// kernel with different sizes (independent solves on concurrent streams).
inline cudaError_t smem_limit_max(const void* kernel) {
  static std::mutex m;
  static std::unordered_set<const void*> done;
  std::lock_guard<std::mutex> guard(m);
  if (done.count(kernel)) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert(kernel);
  return e;
}

typedef double2 cd;
typedef float2 cf;

constexpr int kMaxLayers = 256;
constexpr int kMaxNloc = 118;  // Gauss-Jordan of one Schur complement held in 227 KB of shared memory

// Learned correction network (flat parameter layout shared with the oracle):
// W1 (W, 8, 7) | b1 (W) | W2 (W, W) | b2 (W) | W3 (W, W) | b3 (W) | W4 (8, W) | b4 (8)
constexpr int kNnCin = 8, kNnK1 = 7, kNnW = 256;
constexpr size_t kNnOffW1 = 0;
constexpr size_t kNnOffB1 = kNnOffW1 + (size_t)kNnW * kNnCin * kNnK1;
constexpr size_t kNnOffW2 = kNnOffB1 + kNnW;
constexpr size_t kNnOffB2 = kNnOffW2 + (size_t)kNnW * kNnW;
constexpr size_t kNnOffW3 = kNnOffB2 + kNnW;
constexpr size_t kNnOffB3 = kNnOffW3 + (size_t)kNnW * kNnW;
constexpr size_t kNnOffW4 = kNnOffB3 + kNnW;
constexpr size_t kNnOffB4 = kNnOffW4 + (size_t)kNnCin * kNnW;
constexpr size_t kNnParams = kNnOffB4 + kNnCin;

// Device error word bits (ctx->status on the device)
constexpr int kErrSingular = 1;
constexpr int kErrNumeric = 2;
constexpr int kErrTimeout = 4;
constexpr int kErrArg = 8;

struct LayerInfo {
  int start;    // first extended-grid row of the layer
  int n;        // rows of the layer (n^l)
  int pad_top;  // padded PML rows above local paper row 1
  int pad_bot;
  int nloc;     // rows of the local problem
  int has_top, has_bot;
  int row[4];   // local array row of paper rows 0, 1, n, n+1 (-1 if absent)
  long long sinv_off;  // element offset of Sinv[l][0] in the factor array
  long long coef_off;  // element offset of W[l][0][0] / E[l][0][0]
};

struct Geometry {
  int nt;       // n_t = n_x + 2 n_pml
  int Nz;       // N_z = n_z + 2 n_pml
  int npml;
  int L;
  double h, omega, C;
};

// One output trace of a block-sparse trace operator:
//   out[r] = sum_t sign_t * (B_t (x[in1_t] + x[in2_t]))[r] + sum_e sign_e * src_e[trace_e][r]
struct ApplyTerm {
  int block;  // absolute block index (layer * 16 + jk)
  int in1, in2;  // input traces (in2 = -1: none)
  double sign;
};
struct ApplyRow {
  int out;
  int nterms;
  ApplyTerm t[4];
  int nid;
  int id_src[2];    // 0: the multiplied vector x, 1: the auxiliary vector
  int id_trace[2];
  double id_sign[2];
};

// Extraction task of the offline phase: one layer, a chunk of w source
// columns starting at c0, nk source rows (block indices kk); nk * w == 32.
struct ExtractTask {
  int layer;
  int c0;
  int nk;
  int kk[4];
  int w;
};

// Partitioned low-rank leaf (Section 5.1) and projection task of the PLR apply.
struct PlrLeaf {
  int r0, c0, m, n, rank, kind;  // kind 0: dense, 1: low rank
  long long off;                 // absolute offset in the factor pool:
                                 //   low rank: (U S)^T at off (rank x m), (V^H)^T at off + rank*m (n x rank)
                                 //   dense:    the leaf transposed at off (n x m)
};
struct PlrTask {
  int row, term, leaf;
};

// Tensor-core apply: one output trace of a batched operator (see pt_tc.cu).
struct TcTerm {
  int a_row0;  // first row of the block in the stacked FP16 block tensor (slot * n_t)
  int key;     // staged operand: rows [key * 2S, (key + 1) * 2S) of the stacked operand tensor
};
struct TcRow {
  int out, nterms;
  TcTerm t[4];
  int nid;
  int id_src[2], id_trace[2];
  double id_sign[2];
};
struct TcKey {  // staged input sign * (x[in1] + x[in2])
  int in1, in2;
  double sign;
};

__device__ __forceinline__ cd cmul(cd a, cd b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a * b + c
__device__ __forceinline__ cd cfma(cd a, cd b, cd c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ cd cadd(cd a, cd b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd csub(cd a, cd b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd cscale(cd a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cd cinv(cd a) {
  double d = 1.0 / cabs2(a);
  return make_double2(a.x * d, -a.y * d);
}
__device__ __forceinline__ cf cfmaf(cf a, cf b, cf c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

__device__ __forceinline__ cd shfl_down_cd(cd v, int off) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, off);
  v.y = __shfl_down_sync(0xffffffffu, v.y, off);
  return v;
}
__device__ __forceinline__ cd warp_sum_cd(cd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = cadd(v, shfl_down_cd(v, o));
  return v;
}
__device__ __forceinline__ cf warp_sum_cf(cf v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// PML: alpha = 1 / (1 + i sigma / omega), sigma = (C/delta)(d/delta)^2, d = depth
// into the layer measured from the edge nodes npml-1 and n-npml (Section 2.1).
__device__ __forceinline__ cd pml_alpha(double pos, int n, const Geometry& g) {
  double d = fmax(fmax((double)(g.npml - 1) - pos, pos - (double)(n - g.npml)), 0.0) * g.h;
  double delta = g.npml * g.h;
  double s = (g.C / delta) * (d / delta) * (d / delta) / g.omega;  // sigma / omega
  double den = 1.0 / (1.0 + s * s);
  return make_double2(den, -s * den);
}

}  // namespace pt
