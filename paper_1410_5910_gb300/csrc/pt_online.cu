// Online phase (Algorithm 2) kernels.
//
//  * apply_kernel        block-sparse trace operators of the polarized jump
//                        system (Definition 9 after the permutation P of
//                        Section 3.5): the matvec D + R, the coupling R, one
//                        step of each sweep D_down^{-1} / D_up^{-1}
//                        (Section 4.1).  Each output trace is a sum of at most
//                        four n_t x n_t block products plus identity terms,
//                        described by an ApplyRow table built on the host.
//  * layer_solve_kernel  local solves (H^l)^{-1} with the block factorization
//                        of the offline phase, one thread-block cluster per
//                        (layer, source); forms the interface right-hand side
//                        from N^l f^l (Algorithm 2, "solve local problems")
//                        or rebuilds the volume field from the traces with the
//                        forcing of the PDE form of the discrete GRF (Section 2.3).
//  * GMRES kernels       FP64 dot products, vector updates, norms and the
//                        Givens update of the Hessenberg least squares
//                        (Section 4.2).
#include <cooperative_groups.h>

#include <algorithm>

#include "pt_common.cuh"

namespace cg = cooperative_groups;

namespace pt {

// ---------------------------------------------------------------------------
// block-sparse trace operators
// ---------------------------------------------------------------------------
template <typename BT>
__device__ __forceinline__ cd load_block(const BT* p);
template <>
__device__ __forceinline__ cd load_block<cd>(const cd* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ cd load_block<cf>(const cf* p) {
  cf v = __ldg(p);
  return make_double2(v.x, v.y);
}

// grid (ceil(nt / rows_per_cta), nrows, nsrc), block 256.
// y[s][row.out][r] = sum_t sign_t B_t (x[s][in1] + x[s][in2]) [r] + identity terms.
template <typename BT>
__global__ void __launch_bounds__(256) apply_kernel(int nt, int T4, const ApplyRow* __restrict__ table,
                                                    const BT* __restrict__ blocks, const cd* __restrict__ x,
                                                    const cd* __restrict__ aux, cd* __restrict__ y,
                                                    int rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd* xin = reinterpret_cast<cd*>(smem_raw);  // 4 x nt
  const ApplyRow row = table[blockIdx.y];
  const int s = blockIdx.z;
  const size_t vs = (size_t)T4 * nt;
  const cd* xs = x + s * vs;
  const cd* as = aux ? aux + s * vs : nullptr;
  for (int t = 0; t < row.nterms; ++t) {
    const ApplyTerm tm = row.t[t];
    const cd* a = xs + (size_t)tm.in1 * nt;
    const cd* b = tm.in2 >= 0 ? xs + (size_t)tm.in2 * nt : nullptr;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      cd v = a[k];
      if (b) v = cadd(v, b[k]);
      xin[t * nt + k] = cscale(v, tm.sign);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * rows_per_cta;
  const size_t bsz = (size_t)nt * nt;
  for (int rr = warp; rr < rows_per_cta; rr += 8) {
    const int r = r0 + rr;
    if (r >= nt) break;
    cd acc = make_double2(0, 0);
    for (int t = 0; t < row.nterms; ++t) {
      const BT* B = blocks + (size_t)row.t[t].block * bsz + (size_t)r * nt;
      const cd* xv = xin + t * nt;
      int k = lane;
      for (; k + 96 < nt; k += 128) {
        cd b0 = load_block(B + k), b1 = load_block(B + k + 32), b2 = load_block(B + k + 64), b3 = load_block(B + k + 96);
        acc = cfma(b0, xv[k], acc);
        acc = cfma(b1, xv[k + 32], acc);
        acc = cfma(b2, xv[k + 64], acc);
        acc = cfma(b3, xv[k + 96], acc);
      }
      for (; k < nt; k += 32) acc = cfma(load_block(B + k), xv[k], acc);
    }
    acc = warp_sum_cd(acc);
    if (lane == 0) {
      for (int e = 0; e < row.nid; ++e) {
        const cd* src = row.id_src[e] == 0 ? xs : as;
        acc = cadd(acc, cscale(src[(size_t)row.id_trace[e] * nt + r], row.id_sign[e]));
      }
      y[s * vs + (size_t)row.out * nt + r] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// local solves
// ---------------------------------------------------------------------------
// flag[s * L + l] = 1 when f^l of source s has a non-zero entry
__global__ void layer_nonzero_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cd* __restrict__ f,
                                     int* __restrict__ flag) {
  const LayerInfo L = layers[blockIdx.x];
  const int s = blockIdx.y;
  const cd* fs = f + (size_t)s * g.Nz * g.nt + (size_t)L.start * g.nt;
  int nz = 0;
  for (size_t k = threadIdx.x; k < (size_t)L.n * g.nt; k += blockDim.x) {
    cd v = fs[k];
    nz |= (v.x != 0.0 || v.y != 0.0);
  }
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) flag[s * g.L + blockIdx.x] = nz;
}

constexpr int kSolveCS = 8;                                       // CTAs per cluster
constexpr int kSolveRowsPerCta = (kMaxNloc + kSolveCS - 1) / kSolveCS;  // 15
constexpr int kSolveRW = (kSolveRowsPerCta + 7) / 8;              // rows per warp: 2
constexpr int kSolveCW = (kMaxNloc + 31) / 32;                    // columns per lane: 4

// MODE 0: right-hand side.  out = P b (trace vector), b = (-f, -f_0):
//   down rows of interface l: -N^l_n f, -N^l_{n+1} f; up rows of interface l-1: -N^l_0 f, -N^l_1 f.
// MODE 1: reconstruction.  out = volume field; forcing f^l + (1/h^2)(row 1: +u_0,
//   row 0: -u_1, row n+1: -u_n, row n: +u_{n+1}) with u = u_down + u_up from xtr.
template <int MODE>
__global__ void __cluster_dims__(kSolveCS, 1, 1) __launch_bounds__(256)
    layer_solve_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cd* __restrict__ Sinv,
                       const cd* __restrict__ W, const cd* __restrict__ E, const cd* __restrict__ f,
                       const cd* __restrict__ xtr, cd* __restrict__ Ystore, size_t ystride, cd* __restrict__ out,
                       const int* __restrict__ nzflag) {
  __shared__ __align__(16) cd ybuf[2][kMaxNloc];
  __shared__ __align__(16) cd vloc[kMaxNloc];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int l = blockIdx.x / kSolveCS;
  const int s = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt;
  const int T = 2 * (g.L - 1);
  const size_t T4n = (size_t)2 * T * nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpc = (n + kSolveCS - 1) / kSolveCS;
  const int r0 = rank * rpc, r1 = min(n, r0 + rpc);

  if (MODE == 0 && nzflag[s * g.L + l] == 0) {
    // f^l = 0: the local potentials vanish
    cd* b = out + (size_t)s * T4n;
    for (int k = rank * blockDim.x + threadIdx.x; k < nt; k += kSolveCS * blockDim.x) {
      if (L.has_bot) {
        b[(size_t)(2 * l) * nt + k] = make_double2(0, 0);
        b[(size_t)(2 * l + 1) * nt + k] = make_double2(0, 0);
      }
      if (L.has_top) {
        b[(size_t)(T + 2 * (l - 1)) * nt + k] = make_double2(0, 0);
        b[(size_t)(T + 2 * (l - 1) + 1) * nt + k] = make_double2(0, 0);
      }
    }
    return;  // uniform over the cluster: no cluster barrier has been used
  }

  const cd* fs = f + (size_t)s * g.Nz * nt;
  const cd* xs = (MODE == 1) ? xtr + (size_t)s * T4n : nullptr;
  cd* Y = Ystore + ((size_t)s * g.L + l) * ystride;
  const double ih2 = 1.0 / (g.h * g.h);
  const int nsteps = 2 * nt - 1;

  auto step_col = [&](int st) { return st < nt ? st : (nt - 2 - (st - nt)); };
  auto collapsed = [&](int trace, int i) {  // u = u_down + u_up of trace (0 .. T-1)
    cd a = xs[(size_t)trace * nt + i];
    cd b = xs[(size_t)(T + trace) * nt + i];
    return cadd(a, b);
  };
  auto rhs_val = [&](int i, int r) {
    cd v = make_double2(0, 0);
    if (r >= L.pad_top && r < L.pad_top + L.n) v = fs[(size_t)(L.start + r - L.pad_top) * nt + i];
    if (MODE == 1) {
      if (L.has_top) {
        if (r == L.row[1]) v = cadd(v, cscale(collapsed(2 * (l - 1), i), ih2));
        if (r == L.row[0]) v = csub(v, cscale(collapsed(2 * (l - 1) + 1, i), ih2));
      }
      if (L.has_bot) {
        if (r == L.row[3]) v = csub(v, cscale(collapsed(2 * l, i), ih2));
        if (r == L.row[2]) v = cadd(v, cscale(collapsed(2 * l + 1, i), ih2));
      }
    }
    return v;
  };
  auto emit = [&](int i, int r, cd x) {
    if (MODE == 0) {
      cd* b = out + (size_t)s * T4n;
      cd mx = make_double2(-x.x, -x.y);
      if (L.has_bot) {
        if (r == L.row[2]) b[(size_t)(2 * l) * nt + i] = mx;
        if (r == L.row[3]) b[(size_t)(2 * l + 1) * nt + i] = mx;
      }
      if (L.has_top) {
        if (r == L.row[0]) b[(size_t)(T + 2 * (l - 1)) * nt + i] = mx;
        if (r == L.row[1]) b[(size_t)(T + 2 * (l - 1) + 1) * nt + i] = mx;
      }
    } else {
      if (r >= L.pad_top && r < L.pad_top + L.n)
        out[(size_t)s * g.Nz * nt + (size_t)(L.start + r - L.pad_top) * nt + i] = x;
    }
  };

  // register prefetch of this thread's Sinv entries for the next step
  cd pre[kSolveRW][kSolveCW];
  auto fetch = [&](int st, cd (&dst)[kSolveRW][kSolveCW]) {
    const cd* S = Sinv + L.sinv_off + (size_t)step_col(st) * n * n;
#pragma unroll
    for (int a = 0; a < kSolveRW; ++a) {
      int r = r0 + warp + 8 * a;
#pragma unroll
      for (int c = 0; c < kSolveCW; ++c) {
        int k = lane + 32 * c;
        dst[a][c] = (r < r1 && k < n) ? __ldg(S + (size_t)r * n + k) : make_double2(0, 0);
      }
    }
  };
  fetch(0, pre);
  cluster.sync();  // every CTA of the cluster is resident before remote stores

  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < nt;
    const int i = step_col(st);
    cd cur[kSolveRW][kSolveCW];
#pragma unroll
    for (int a = 0; a < kSolveRW; ++a)
#pragma unroll
      for (int c = 0; c < kSolveCW; ++c) cur[a][c] = pre[a][c];
    // v = f_i - W_i o y_{i-1}   (forward)   |   v = E_i o x_{i+1}   (backward)
    const cd* prev = ybuf[(i + 1) & 1];  // y_{i-1} (forward) or x_{i+1} (backward): the other buffer
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      cd v;
      if (fwd) {
        v = rhs_val(i, r);
        if (i > 0) v = csub(v, cmul(W[L.coef_off + (size_t)i * n + r], prev[r]));
      } else {
        v = cmul(E[L.coef_off + (size_t)i * n + r], prev[r]);
      }
      vloc[r] = v;
    }
    __syncthreads();
    if (st + 1 < nsteps) fetch(st + 1, pre);
    cd* ycur = ybuf[i & 1];
#pragma unroll
    for (int a = 0; a < kSolveRW; ++a) {
      const int r = r0 + warp + 8 * a;
      cd acc = make_double2(0, 0);
#pragma unroll
      for (int c = 0; c < kSolveCW; ++c) {
        int k = lane + 32 * c;
        if (k < n) acc = cfma(cur[a][c], vloc[k], acc);
      }
      acc = warp_sum_cd(acc);
      if (r < r1 && lane == 0) {
        cd val;
        if (fwd) {
          val = acc;
          Y[(size_t)i * n + r] = acc;
        } else {
          val = csub(Y[(size_t)i * n + r], acc);
        }
        for (int q = 0; q < kSolveCS; ++q) cluster.map_shared_rank(ycur, q)[r] = val;
        if (!fwd || i == nt - 1) emit(i, r, val);
      }
    }
    cluster.sync();
  }
}

// ---------------------------------------------------------------------------
// GMRES (FP64).  Basis layout V[j][s][N], N = 4 (L-1) n_t complex entries.
// ---------------------------------------------------------------------------
constexpr int kDotThreads = 256;
constexpr int kDotChunk = 4096;  // entries per CTA

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

// nrm[s] = ||w_s||, optional H[s][row][col] = nrm; dst_s = w_s / nrm (0 when nrm ~ 0).  One CTA per source.
__global__ void __launch_bounds__(1024) norm_scale_kernel(const cd* __restrict__ w, size_t N, double* __restrict__ nrm,
                                                          cd* __restrict__ H, int hrows, int hcols, int row, int col,
                                                          cd* __restrict__ dst, size_t dst_stride) {
  const int s = blockIdx.x;
  const cd* ws = w + (size_t)s * N;
  double acc = 0.0;
  for (size_t k = threadIdx.x; k < N; k += blockDim.x) acc = fma(ws[k].x, ws[k].x, fma(ws[k].y, ws[k].y, acc));
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  __shared__ double s_n;
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      s_n = sqrt(v);
      if (nrm) nrm[s] = s_n;
      if (H) H[((size_t)s * hrows + row) * hcols + col] = make_double2(s_n, 0.0);
    }
  }
  __syncthreads();
  if (dst) {
    const double nv = s_n;
    const double inv = nv > 1e-300 ? 1.0 / nv : 0.0;
    for (size_t k = threadIdx.x; k < N; k += blockDim.x) dst[(size_t)s * dst_stride + k] = cscale(ws[k], inv);
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
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_apply(int nt, int T4, const ApplyRow* table, int nrows, bool fp32, const void* blocks,
                         const cd* x, const cd* aux, cd* y, int nsrc, int rows_per_cta, cudaStream_t s) {
  size_t smem = 4ull * nt * sizeof(cd);
  dim3 grid((nt + rows_per_cta - 1) / rows_per_cta, nrows, nsrc);
  if (fp32) {
    cudaFuncSetAttribute(apply_kernel<cf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_kernel<cf><<<grid, 256, smem, s>>>(nt, T4, table, (const cf*)blocks, x, aux, y, rows_per_cta);
  } else {
    cudaFuncSetAttribute(apply_kernel<cd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_kernel<cd><<<grid, 256, smem, s>>>(nt, T4, table, (const cd*)blocks, x, aux, y, rows_per_cta);
  }
  return cudaGetLastError();
}

cudaError_t launch_layer_nonzero(const Geometry& g, const LayerInfo* layers, const cd* f, int* flag, int nsrc,
                                 cudaStream_t s) {
  layer_nonzero_kernel<<<dim3(g.L, nsrc), 256, 0, s>>>(g, layers, f, flag);
  return cudaGetLastError();
}

cudaError_t launch_layer_solve(int mode, const Geometry& g, const LayerInfo* layers, const cd* Sinv, const cd* W,
                               const cd* E, const cd* f, const cd* xtr, cd* Y, size_t ystride, cd* out,
                               const int* flag, int nsrc, cudaStream_t s) {
  dim3 grid(kSolveCS * g.L, nsrc);
  if (mode == 0)
    layer_solve_kernel<0><<<grid, 256, 0, s>>>(g, layers, Sinv, W, E, f, xtr, Y, ystride, out, flag);
  else
    layer_solve_kernel<1><<<grid, 256, 0, s>>>(g, layers, Sinv, W, E, f, xtr, Y, ystride, out, flag);
  return cudaGetLastError();
}

int dot_chunks(size_t N) { return (int)((N + kDotChunk - 1) / kDotChunk); }

cudaError_t launch_dots(const cd* V, int nsrc, size_t N, const cd* w, int nvec, cd* partial, cd* coef,
                        int coef_stride, cd* H, int hrows, int hcols, int col, cudaStream_t s) {
  int nch = dot_chunks(N);
  dots_kernel<<<dim3(nch, nvec, nsrc), kDotThreads, 0, s>>>(V, nsrc, N, w, nvec, nch, partial);
  dots_finalize_kernel<<<dim3(nvec, nsrc), 32, 0, s>>>(partial, nvec, nch, coef, coef_stride, H, hrows, hcols, col);
  return cudaGetLastError();
}

cudaError_t launch_update(const cd* V, int nsrc, size_t N, cd* w, int nvec, const cd* coef, int coef_stride,
                          cudaStream_t s) {
  int gx = (int)std::min<size_t>((N + 1023) / 1024, 1024);
  update_kernel<<<dim3(gx, nsrc), 256, 0, s>>>(V, nsrc, N, w, nvec, coef, coef_stride);
  return cudaGetLastError();
}

cudaError_t launch_norm_scale(const cd* w, size_t N, int nsrc, double* nrm, cd* H, int hrows, int hcols, int row,
                              int col, cd* dst, size_t dst_stride, cudaStream_t s) {
  norm_scale_kernel<<<nsrc, 1024, 0, s>>>(w, N, nrm, H, hrows, hcols, row, col, dst, dst_stride);
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
