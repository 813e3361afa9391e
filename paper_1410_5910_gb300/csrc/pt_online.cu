// GMRES kernels of the online phase (Section 4.2), FP64: dot products with a
// fixed-order two-stage reduction, vector updates, norms with scaling, the
// Givens update of the Hessenberg least squares, the triangular solve and
// the combination of the preconditioned Krylov vectors (flexible GMRES).
#include <algorithm>

#include "pt_common.cuh"

namespace pt {

// ---------------------------------------------------------------------------
// GMRES (FP64).  Basis layout V[j][s][N], N = 4 (L-1) n_t complex entries.
// ---------------------------------------------------------------------------
constexpr int kDotThreads = 256;
constexpr int kDotChunk = 1024;  // entries per CTA: the FP64 work of a reduction spread over the SMs

// partial[(s * nvec + j) * nchunks + c] = sum_{k in chunk c} conj(V_j[s][k]) w[s][k]
__global__ void __launch_bounds__(kDotThreads) dots_kernel(const cd* __restrict__ V, int nsrc, size_t N,
                                                           const cd* __restrict__ w, int nvec, int nchunks,
                                                           cd* __restrict__ partial) {
  const int c = blockIdx.x, j = blockIdx.y, s = blockIdx.z;
  const cd* v = V + ((size_t)j * nsrc + s) * N;
  const cd* ws = w + (size_t)s * N;
  cd acc = make_double2(0, 0);
  size_t k0 = (size_t)c * kDotChunk, k1 = min(N, k0 + kDotChunk);
  for (size_t k = k0 + threadIdx.x; k < k1; k += kDotThreads) {
    cd a = v[k], b = ws[k];
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
  }
  __shared__ cd red[kDotThreads / 32];
  acc = warp_sum_cd(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    cd v2 = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : make_double2(0, 0);
    v2 = warp_sum_cd(v2);
    if (threadIdx.x == 0) partial[((size_t)s * nvec + j) * nchunks + c] = v2;
  }
}

// coef[s][j] = sum_c partial; H[s][j][col] += coef (when H != null).  grid (nvec, nsrc), block 32.
__global__ void dots_finalize_kernel(const cd* __restrict__ partial, int nvec, int nchunks, cd* __restrict__ coef,
                                     int coef_stride, cd* __restrict__ H, int hrows, int hcols, int col) {
  const int j = blockIdx.x, s = blockIdx.y;
  cd acc = make_double2(0, 0);
  for (int c = threadIdx.x; c < nchunks; c += 32) acc = cadd(acc, partial[((size_t)s * nvec + j) * nchunks + c]);
  acc = warp_sum_cd(acc);
  if (threadIdx.x == 0) {
    coef[(size_t)s * coef_stride + j] = acc;
    if (H) {
      cd* h = H + ((size_t)s * hrows + j) * hcols + col;
      *h = cadd(*h, acc);
    }
  }
}

// w[s][k] -= sum_j coef[s][j] V_j[s][k].  grid (ceil(N/1024), nsrc), block 256
__global__ void update_kernel(const cd* __restrict__ V, int nsrc, size_t N, cd* __restrict__ w, int nvec,
                              const cd* __restrict__ coef, int coef_stride) {
  const int s = blockIdx.y;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
    cd acc = w[(size_t)s * N + k];
    for (int j = 0; j < nvec; ++j) {
      cd a = coef[(size_t)s * coef_stride + j];
      cd v = V[((size_t)j * nsrc + s) * N + k];
      acc = csub(acc, cmul(a, v));
    }
    w[(size_t)s * N + k] = acc;
  }
}

// nrm[s] = ||w_s||, optional H[s][row][col] = nrm; dst_s = w_s / nrm (0 when nrm ~ 0).
// Two passes over chunks of kNormChunk entries: per-chunk sums of squares, then every
// chunk's CTA forms the same total (the partials summed in a fixed order), and scales
// its chunk.  A single CTA per source would keep the whole vector's FP64 arithmetic on
// one SM's FP64 pipe (2 lanes per clock on GB300).
constexpr int kNormChunk = 1024;
constexpr int kNormThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kNormThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();  // red is reused by the caller's next reduction
  return t;
}

__global__ void __launch_bounds__(kNormThreads) norm_partial_kernel(const cd* __restrict__ w, size_t N, int nb,
                                                                     double* __restrict__ part) {
  const int b = blockIdx.x, s = blockIdx.y;
  const cd* ws = w + (size_t)s * N;
  const size_t k0 = (size_t)b * kNormChunk, k1 = min(N, k0 + kNormChunk);
  double acc = 0.0;
  for (size_t k = k0 + threadIdx.x; k < k1; k += kNormThreads) acc = fma(ws[k].x, ws[k].x, fma(ws[k].y, ws[k].y, acc));
  __shared__ double red[32];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)s * nb + b] = acc;
}

__global__ void __launch_bounds__(kNormThreads) norm_finish_kernel(const cd* __restrict__ w, size_t N, int nb,
                                                                    const double* __restrict__ part,
                                                                    double* __restrict__ nrm, cd* __restrict__ H,
                                                                    int hrows, int hcols, int row, int col,
                                                                    cd* __restrict__ dst, size_t dst_stride) {
  const int b = blockIdx.x, s = blockIdx.y;
  double acc = 0.0;
  for (int c = threadIdx.x; c < nb; c += kNormThreads) acc += part[(size_t)s * nb + c];
  __shared__ double red[32];
  const double nv = sqrt(block_sum(acc, red));
  if (b == 0 && threadIdx.x == 0) {
    if (nrm) nrm[s] = nv;
    if (H) H[((size_t)s * hrows + row) * hcols + col] = make_double2(nv, 0.0);
  }
  if (dst) {
    const double inv = nv > 1e-300 ? 1.0 / nv : 0.0;
    const cd* ws = w + (size_t)s * N;
    const size_t k0 = (size_t)b * kNormChunk, k1 = min(N, k0 + kNormChunk);
    for (size_t k = k0 + threadIdx.x; k < k1; k += kNormThreads) dst[(size_t)s * dst_stride + k] = cscale(ws[k], inv);
  }
}

// Givens update of column j of the Hessenberg matrix of each source (Section 4.2).
// H[s] is (m+1) x m row-major; cs[s][m], sn[s][m]; g[s][m+1]; resid[s] = |g_{j+1}|.
__global__ void givens_kernel(int nsrc, int m, int j, cd* __restrict__ H, double* __restrict__ cs,
                              cd* __restrict__ sn, cd* __restrict__ gv, double* __restrict__ resid) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsrc) return;
  cd* Hs = H + (size_t)s * (m + 1) * m;
  double* c = cs + (size_t)s * m;
  cd* sv = sn + (size_t)s * m;
  cd* g = gv + (size_t)s * (m + 1);
  for (int i = 0; i < j; ++i) {
    cd a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
    cd t = cadd(cscale(a, c[i]), cmul(sv[i], b));
    cd snc = make_double2(sv[i].x, -sv[i].y);
    cd u = csub(cscale(b, c[i]), cmul(snc, a));
    Hs[i * m + j] = t;
    Hs[(i + 1) * m + j] = u;
  }
  cd a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
  double na = sqrt(cabs2(a)), nb = sqrt(cabs2(b));
  double cc;
  cd ss;
  if (nb == 0.0) {
    cc = 1.0;
    ss = make_double2(0, 0);
  } else if (na == 0.0) {
    cc = 0.0;
    ss = make_double2(b.x / nb, -b.y / nb);
  } else {
    double tt = hypot(na, nb);
    cc = na / tt;
    cd ph = make_double2(a.x / na, a.y / na);
    ss = cscale(cmul(ph, make_double2(b.x, -b.y)), 1.0 / tt);
  }
  c[j] = cc;
  sv[j] = ss;
  Hs[j * m + j] = cadd(cscale(a, cc), cmul(ss, b));
  Hs[(j + 1) * m + j] = make_double2(0, 0);
  cd gj = g[j];
  cd ssc = make_double2(ss.x, -ss.y);
  cd gn = cmul(ssc, gj);
  g[j + 1] = make_double2(-gn.x, -gn.y);
  g[j] = cscale(gj, cc);
  resid[s] = sqrt(cabs2(g[j + 1]));
}

// y = R^{-1} g on the leading k_s x k_s triangle (k_s = kk[s]); one thread per source.
__global__ void lsq_solve_kernel(int nsrc, int m, const int* __restrict__ kk, const cd* __restrict__ H,
                                 const cd* __restrict__ gv, cd* __restrict__ y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsrc) return;
  const cd* Hs = H + (size_t)s * (m + 1) * m;
  const cd* g = gv + (size_t)s * (m + 1);
  cd* ys = y + (size_t)s * (m + 1);
  const int k = kk[s];
  for (int i = k - 1; i >= 0; --i) {
    cd acc = g[i];
    for (int q = i + 1; q < k; ++q) acc = csub(acc, cmul(Hs[i * m + q], ys[q]));
    cd d = Hs[i * m + i];
    ys[i] = (cabs2(d) > 0) ? cmul(acc, cinv(d)) : make_double2(0, 0);
  }
  for (int i = k; i <= m; ++i) ys[i] = make_double2(0, 0);
}

// x[s] += sum_{j < kk[s]} y[s][j] Z_j[s]   grid (ceil(N/1024), nsrc)
__global__ void combine_kernel(const cd* __restrict__ Z, int nsrc, size_t N, const cd* __restrict__ y, int m,
                               const int* __restrict__ kk, cd* __restrict__ x) {
  const int s = blockIdx.y;
  const int k = kk[s];
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < N; q += (size_t)gridDim.x * blockDim.x) {
    cd acc = x[(size_t)s * N + q];
    for (int j = 0; j < k; ++j) acc = cadd(acc, cmul(y[(size_t)s * (m + 1) + j], Z[((size_t)j * nsrc + s) * N + q]));
    x[(size_t)s * N + q] = acc;
  }
}

// z = a - b (elementwise), n entries
__global__ void sub_kernel(const cd* __restrict__ a, const cd* __restrict__ b, cd* __restrict__ z, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    z[k] = csub(a[k], b[k]);
}

// ---------------------------------------------------------------------------
// FP64 residual of the global discrete Helmholtz equation (Section 2.1)
// ---------------------------------------------------------------------------
constexpr int kVresBlocks = 512;

// partial[(s * kVresBlocks + b) * 2 + {0, 1}] = sum over the block's points of |f - H u|^2 and |f|^2
__global__ void __launch_bounds__(256) volres_kernel(Geometry g, const double* __restrict__ c_ext,
                                                     const cd* __restrict__ f, const cd* __restrict__ u,
                                                     double* __restrict__ partial) {
  const int s = blockIdx.y;
  const size_t np = (size_t)g.Nz * g.nt;
  const cd* us = u + s * np;
  const cd* fs = f + s * np;
  const double ih2 = 1.0 / (g.h * g.h);
  double rr = 0.0, ff = 0.0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < np; idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx / g.nt), p = (int)(idx - (size_t)q * g.nt);
    const cd ax = pml_alpha(p, g.nt, g), axp = pml_alpha(p + 0.5, g.nt, g), axm = pml_alpha(p - 0.5, g.nt, g);
    const cd az = pml_alpha(q, g.Nz, g), azp = pml_alpha(q + 0.5, g.Nz, g), azm = pml_alpha(q - 0.5, g.Nz, g);
    const double c = c_ext[idx];
    const double m = 1.0 / (c * c);
    const cd sx = cmul(ax, cadd(axp, axm)), sz = cmul(az, cadd(azp, azm));
    const cd center = make_double2((sx.x + sz.x) * ih2 - g.omega * g.omega * m, (sx.y + sz.y) * ih2);
    cd hu = cmul(center, us[idx]);
    if (p > 0) hu = cadd(hu, cmul(cscale(cmul(ax, axm), -ih2), us[idx - 1]));
    if (p < g.nt - 1) hu = cadd(hu, cmul(cscale(cmul(ax, axp), -ih2), us[idx + 1]));
    if (q > 0) hu = cadd(hu, cmul(cscale(cmul(az, azm), -ih2), us[idx - g.nt]));
    if (q < g.Nz - 1) hu = cadd(hu, cmul(cscale(cmul(az, azp), -ih2), us[idx + g.nt]));
    const cd r = csub(fs[idx], hu);
    rr += cabs2(r);
    ff += cabs2(fs[idx]);
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    ff += __shfl_down_sync(0xffffffffu, ff, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = ff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partial[((size_t)s * gridDim.x + blockIdx.x) * 2] = a;
    partial[((size_t)s * gridDim.x + blockIdx.x) * 2 + 1] = b;
  }
}

__global__ void volres_final_kernel(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  const int s = blockIdx.x;
  double a = 0, b = 0;
  for (int k = threadIdx.x; k < nblk; k += 32) {
    a += partial[((size_t)s * nblk + k) * 2];
    b += partial[((size_t)s * nblk + k) * 2 + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (threadIdx.x == 0) out[s] = b > 0 ? sqrt(a / b) : sqrt(a);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int dot_chunks(size_t N) { return (int)((N + kDotChunk - 1) / kDotChunk); }

// work: at least nsrc + 2 * nsrc * 512 doubles; out = work[0 .. nsrc)
cudaError_t launch_volume_residual(const Geometry& g, const double* c_ext, const cd* f, const cd* u, int nsrc,
                                   double* work, cudaStream_t s) {
  double* partial = work + nsrc;
  volres_kernel<<<dim3(kVresBlocks, nsrc), 256, 0, s>>>(g, c_ext, f, u, partial);
  volres_final_kernel<<<nsrc, 32, 0, s>>>(partial, kVresBlocks, work);
  return cudaGetLastError();
}

cudaError_t launch_dots(const cd* V, int nsrc, size_t N, const cd* w, int nvec, cd* partial, cd* coef,
                        int coef_stride, cd* H, int hrows, int hcols, int col, cudaStream_t s) {
  int nch = dot_chunks(N);
  dots_kernel<<<dim3(nch, nvec, nsrc), kDotThreads, 0, s>>>(V, nsrc, N, w, nvec, nch, partial);
  dots_finalize_kernel<<<dim3(nvec, nsrc), 32, 0, s>>>(partial, nvec, nch, coef, coef_stride, H, hrows, hcols, col);
  return cudaGetLastError();
}

cudaError_t launch_update(const cd* V, int nsrc, size_t N, cd* w, int nvec, const cd* coef, int coef_stride,
                          cudaStream_t s) {
  int gx = (int)std::min<size_t>((N + 255) / 256, 4096);  // one entry per thread: the FP64 updates on every SM
  update_kernel<<<dim3(gx, nsrc), 256, 0, s>>>(V, nsrc, N, w, nvec, coef, coef_stride);
  return cudaGetLastError();
}

// part: scratch of nsrc * ceil(N / kNormChunk) doubles
cudaError_t launch_norm_scale(const cd* w, size_t N, int nsrc, double* nrm, cd* H, int hrows, int hcols, int row,
                              int col, cd* dst, size_t dst_stride, double* part, cudaStream_t s) {
  const int nb = (int)((N + kNormChunk - 1) / kNormChunk);
  norm_partial_kernel<<<dim3(nb, nsrc), kNormThreads, 0, s>>>(w, N, nb, part);
  norm_finish_kernel<<<dim3(dst ? nb : 1, nsrc), kNormThreads, 0, s>>>(w, N, nb, part, nrm, H, hrows, hcols, row, col,
                                                                       dst, dst_stride);
  return cudaGetLastError();
}

cudaError_t launch_givens(int nsrc, int m, int j, cd* H, double* cs, cd* sn, cd* g, double* resid, cudaStream_t s) {
  givens_kernel<<<(nsrc + 63) / 64, 64, 0, s>>>(nsrc, m, j, H, cs, sn, g, resid);
  return cudaGetLastError();
}

cudaError_t launch_lsq_combine(int nsrc, int m, const int* kk, const cd* H, const cd* g, cd* y, const cd* Z,
                               size_t N, cd* x, cudaStream_t s) {
  lsq_solve_kernel<<<(nsrc + 63) / 64, 64, 0, s>>>(nsrc, m, kk, H, g, y);
  int gx = (int)std::min<size_t>((N + 1023) / 1024, 1024);
  combine_kernel<<<dim3(gx, nsrc), 256, 0, s>>>(Z, nsrc, N, y, m, kk, x);
  return cudaGetLastError();
}

cudaError_t launch_sub(const cd* a, const cd* b, cd* z, size_t n, cudaStream_t s) {
  int gx = (int)std::min<size_t>((n + 1023) / 1024, 2048);
  sub_kernel<<<gx, 256, 0, s>>>(a, b, z, n);
  return cudaGetLastError();
}

}  // namespace pt
