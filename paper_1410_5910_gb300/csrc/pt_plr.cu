// Partitioned low-rank (PLR) interface blocks (Section 5.1).
//
// Compression (Algorithm 5), offline, FP64: one CTA per block walks the
// quadtree with an explicit stack.  At a node M (m x n) it estimates the
// leading r_max + 1 singular values with a randomized SVD (Section 7.1 uses a
// randomized SVD): Y = M Omega with k = r_max + 1 + p Gaussian columns, one
// power iteration, Q = orth(Y), B^H = M^H Q = Q2 R2 (QR), and a one-sided
// Jacobi SVD of the small R2^H = U S V^H, so that M ~ (Q U) S (Q2 V)^H.  If
// sigma_{r_max+1} < eps sigma_1(block) the node becomes a leaf storing
// U S (m x r) and V^H (r x n), r = #{sigma >= eps sigma_1}, or a dense leaf
// when r (m + n) >= m n or min(m, n) <= r_max; otherwise it splits 2 x 2
// (first half ceil(m/2)).
//
// Application (Algorithm 6 in the flattened "sparse factorization" form):
// plr_project_kernel computes t = V^H x_cols for every low-rank leaf of every
// block term of an operator table (one lane per rank index); plr_expand_kernel
// sums, per tile of 32 output rows, the dense-leaf products and U S t over the
// leaves that cover the tile (one lane per row, warps take whole leaves, a
// shared-memory sum across warps), plus the identity terms.  All factors are
// stored transposed so that both phases read them with unit stride across
// lanes and need no shuffle reductions.
#include <algorithm>

#include "pt_common.cuh"

namespace pt {

constexpr int kPlrK = 48;          // sketch width limit: r_max + 1 + oversampling
constexpr int kPlrThreads = 256;
constexpr int kPlrStack = 96;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
// complex standard Gaussian from a counter (Box-Muller on two 53-bit uniforms)
__device__ cd gauss_c(unsigned long long key) {
  unsigned long long a = mix64(key), b = mix64(key ^ 0x5851f42d4c957f2dull);
  double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
  double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
  double rr = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return make_double2(rr * cs, rr * sn);
}
__device__ __forceinline__ cd conjd(cd a) { return make_double2(a.x, -a.y); }

// out[i][c] = sum_j A(i, j) B[j][c], A(i, j) = M[i*lda + j] (trans = 0) or conj(M[j*lda + i]) (trans = 1)
__device__ void cta_gemm(int rows, int inner, int k, const cd* M, int lda, bool trans, const cd* B, int ldb, cd* out,
                         int ldo) {
  for (int q = threadIdx.x; q < rows * k; q += blockDim.x) {
    const int i = q / k, c = q - (q / k) * k;
    cd acc = make_double2(0, 0);
    if (!trans) {
      const cd* a = M + (size_t)i * lda;
      for (int j = 0; j < inner; ++j) acc = cfma(a[j], B[(size_t)j * ldb + c], acc);
    } else {
      for (int j = 0; j < inner; ++j) acc = cfma(conjd(M[(size_t)j * lda + i]), B[(size_t)j * ldb + c], acc);
    }
    out[(size_t)i * ldo + c] = acc;
  }
  __syncthreads();
}

// Classical Gram-Schmidt twice on the k columns of X (rows x k, row stride ld).
// R (k x k, optional) receives the triangular factor.  Columns whose norm
// collapses below 1e-13 of their original norm are set to zero.
__device__ void cta_orth(int rows, int k, cd* X, int ld, cd* R, cd* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (R)
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) R[q] = make_double2(0, 0);
  __syncthreads();
  for (int c = 0; c < k; ++c) {
    // original norm^2
    double n0 = 0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) n0 += cabs2(X[(size_t)i * ld + c]);
    for (int o = 16; o > 0; o >>= 1) n0 += __shfl_down_sync(0xffffffffu, n0, o);
    if (lane == 0) red[warp].x = n0;
    __syncthreads();
    double norm0 = 0;
    for (int w = 0; w < nw; ++w) norm0 += red[w].x;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      // d_a = X_a^H X_c for a < c (warp per a)
      for (int a = warp; a < c; a += nw) {
        cd d = make_double2(0, 0);
        for (int i = lane; i < rows; i += 32) d = cfma(conjd(X[(size_t)i * ld + a]), X[(size_t)i * ld + c], d);
        d = warp_sum_cd(d);
        if (lane == 0) red[32 + a] = d;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        cd v = X[(size_t)i * ld + c];
        for (int a = 0; a < c; ++a) v = csub(v, cmul(red[32 + a], X[(size_t)i * ld + a]));
        X[(size_t)i * ld + c] = v;
      }
      if (R && threadIdx.x < c) R[threadIdx.x * k + c] = cadd(R[threadIdx.x * k + c], red[32 + threadIdx.x]);
      __syncthreads();
    }
    double nn = 0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) nn += cabs2(X[(size_t)i * ld + c]);
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
    if (lane == 0) red[warp].x = nn;
    __syncthreads();
    double nrm2 = 0;
    for (int w = 0; w < nw; ++w) nrm2 += red[w].x;
    __syncthreads();
    const double nrm = sqrt(nrm2);
    const bool dead = !(nrm > 1e-13 * sqrt(norm0)) || nrm == 0.0;
    const double inv = dead ? 0.0 : 1.0 / nrm;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) X[(size_t)i * ld + c] = cscale(X[(size_t)i * ld + c], inv);
    if (R && threadIdx.x == 0) R[c * k + c] = make_double2(dead ? 0.0 : nrm, 0.0);
    __syncthreads();
  }
}

// One-sided (Hestenes) Jacobi SVD of A (k x k, row-major, in shared memory):
// A V = U S.  On return A holds U S column-scaled (columns are U_j sigma_j),
// V the right vectors, sig the column norms.  Warp 0 does the work.
__device__ void warp_jacobi(int k, cd* A, cd* V, double* sig) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  for (int q = lane; q < k * k; q += 32) V[q] = make_double2((q / k) == (q % k) ? 1.0 : 0.0, 0.0);
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k - 1; ++p) {
      for (int q = p + 1; q < k; ++q) {
        double al = 0, be = 0;
        cd ga = make_double2(0, 0);
        for (int i = lane; i < k; i += 32) {
          cd ap = A[i * k + p], aq = A[i * k + q];
          al += cabs2(ap);
          be += cabs2(aq);
          ga = cfma(conjd(ap), aq, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
        }
        const double g = sqrt(cabs2(ga));
        if (!(g > 1e-15 * sqrt(al * be)) || g == 0.0) continue;
        off = fmax(off, g / sqrt(al * be));
        const double zeta = (al - be) / (2.0 * g);
        const double t = -(zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        const cd e = make_double2(ga.x / g, ga.y / g);  // e^{i phi}
        // [a_p', a_q'] = [a_p, a_q] [[c, s e], [-s conj(e), c]]
        for (int i = lane; i < k; i += 32) {
          cd ap = A[i * k + p], aq = A[i * k + q];
          A[i * k + p] = csub(cscale(ap, c), cscale(cmul(conjd(e), aq), s));
          A[i * k + q] = cadd(cscale(cmul(e, ap), s), cscale(aq, c));
          cd vp = V[i * k + p], vq = V[i * k + q];
          V[i * k + p] = csub(cscale(vp, c), cscale(cmul(conjd(e), vq), s));
          V[i * k + q] = cadd(cscale(cmul(e, vp), s), cscale(vq, c));
        }
        __syncwarp();
      }
    }
    if (off < 1e-15) break;
  }
  for (int j = lane; j < k; j += 32) {
    double s2 = 0;
    for (int i = 0; i < k; ++i) s2 += cabs2(A[i * k + j]);
    sig[j] = sqrt(s2);
  }
  __syncwarp();
}

// A dense leaf: its entries copied transposed (n x m) into the pool, so that the
// apply reads them with unit stride across the lanes that own the rows.
__device__ void dense_leaf(const cd* M, int nt, int r0, int c0, int m, int n, cd* P0, size_t pool_base, PlrLeaf* LV,
                           int& nleaf, long long& pool_off) {
  const long long off = pool_off;
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int j = e / m, i = e - (e / m) * m;
    P0[off + e] = M[(size_t)i * nt + j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    LV[nleaf] = PlrLeaf{r0, c0, m, n, 0, 0, (long long)pool_base + off};
    nleaf++;
    pool_off = off + (long long)m * n;
  }
  __syncthreads();
}

// Persistent over blocks.  Dynamic shared memory: Jacobi A and V (kPlrK^2 each).
__global__ void __launch_bounds__(kPlrThreads) plr_compress_kernel(
    int nt, const cd* __restrict__ blocks, const int* __restrict__ block_ids, int nblk, int rmax, double eps,
    int oversample, cd* __restrict__ scratch, size_t scratch_per_cta, PlrLeaf* __restrict__ leaves, int cap,
    int* __restrict__ nleaves, cd* __restrict__ pool, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd* JA = reinterpret_cast<cd*>(smem_raw);
  cd* JV = JA + kPlrK * kPlrK;
  __shared__ cd red[32 + kPlrK];
  __shared__ double sig[kPlrK];
  __shared__ int perm[kPlrK];
  __shared__ int4 stack[kPlrStack];
  __shared__ int s_sp, s_nleaf;
  __shared__ long long s_pool;
  __shared__ double s_sigma1;
  const size_t S = (size_t)nt * kPlrK;
  cd* Om = scratch + blockIdx.x * scratch_per_cta;
  cd* Y = Om + S;
  cd* Zt = Y + S;
  cd* Bt = Zt + S;
  cd* R2 = Bt + S;  // k x k

  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const cd* M0 = blocks + (size_t)block_ids[b] * nt * nt;
    cd* P0 = pool + (size_t)b * nt * nt;
    PlrLeaf* LV = leaves + (size_t)b * cap;
    if (threadIdx.x == 0) {
      s_sp = 1;
      stack[0] = make_int4(0, 0, nt, nt);
      s_nleaf = 0;
      s_pool = 0;
      s_sigma1 = -1.0;
    }
    __syncthreads();
    while (true) {
      __syncthreads();
      if (s_sp == 0) break;  // uniform: every thread reads s_sp after the barrier
      const int4 nd = stack[s_sp - 1];
      const bool full = s_nleaf + 4 >= cap || s_sp - 1 + 4 > kPlrStack;
      const bool rooted = s_sigma1 > 0;
      __syncthreads();  // everyone has read the stack top before it is popped
      if (threadIdx.x == 0) s_sp--;
      const int r0 = nd.x, c0 = nd.y, m = nd.z, n = nd.w;
      const cd* M = M0 + (size_t)r0 * nt + c0;
      const bool small = min(m, n) <= rmax;
      if (small || (full && rooted)) {
        dense_leaf(M, nt, r0, c0, m, n, P0, (size_t)b * nt * nt, LV, s_nleaf, s_pool);
        continue;
      }
      const int k = min(min(rmax + 1 + oversample, kPlrK), min(m, n));
      // ---- randomized range finder with one power iteration
      for (int q = threadIdx.x; q < n * k; q += blockDim.x) {
        const int j = q / k, c = q - (q / k) * k;
        Om[(size_t)j * kPlrK + c] =
            gauss_c(((unsigned long long)b << 40) ^ ((unsigned long long)(r0 * 4099 + c0) << 20) ^ (unsigned)(j * kPlrK + c));
      }
      __syncthreads();
      cta_gemm(m, n, k, M, nt, false, Om, kPlrK, Y, kPlrK);    // Y = M Omega
      cta_orth(m, k, Y, kPlrK, nullptr, red);
      cta_gemm(n, m, k, M, nt, true, Y, kPlrK, Zt, kPlrK);     // Z = M^H Y
      cta_orth(n, k, Zt, kPlrK, nullptr, red);
      cta_gemm(m, n, k, M, nt, false, Zt, kPlrK, Y, kPlrK);    // Y = M Z
      cta_orth(m, k, Y, kPlrK, nullptr, red);                  // Q = Y
      cta_gemm(n, m, k, M, nt, true, Y, kPlrK, Bt, kPlrK);     // B^H = M^H Q
      cta_orth(n, k, Bt, kPlrK, R2, red);                      // B^H = Q2 R2
      // A = R2^H (k x k) into shared memory
      for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
        const int i = q / k, j = q - (q / k) * k;
        JA[i * k + j] = conjd(R2[j * k + i]);
      }
      __syncthreads();
      warp_jacobi(k, JA, JV, sig);
      __syncthreads();
      if (threadIdx.x == 0) {
        // sort singular values descending (selection over k <= 48)
        for (int j = 0; j < k; ++j) perm[j] = j;
        for (int a = 0; a < k; ++a) {
          int best = a;
          for (int j = a + 1; j < k; ++j)
            if (sig[perm[j]] > sig[perm[best]]) best = j;
          int t = perm[a];
          perm[a] = perm[best];
          perm[best] = t;
        }
        if (s_sigma1 < 0) s_sigma1 = sig[perm[0]];
      }
      __syncthreads();
      const double thr = eps * s_sigma1;
      const bool leaf = (rmax >= k) || (sig[perm[rmax]] < thr);
      if (!leaf) {
        if (threadIdx.x == 0) {
          const int mh = (m + 1) / 2, nh = (n + 1) / 2;
          // push in reverse so that children are processed in (0,0), (0,1), (1,0), (1,1) order
          stack[s_sp++] = make_int4(r0 + mh, c0 + nh, m - mh, n - nh);
          stack[s_sp++] = make_int4(r0 + mh, c0, m - mh, nh);
          stack[s_sp++] = make_int4(r0, c0 + nh, mh, n - nh);
          stack[s_sp++] = make_int4(r0, c0, mh, nh);
        }
        __syncthreads();
        continue;
      }
      int r = 0;
      for (int j = 0; j < k && j < rmax; ++j)
        if (sig[perm[j]] >= thr) r = j + 1;
      if ((long long)r * (m + n) >= (long long)m * n) {
        dense_leaf(M, nt, r0, c0, m, n, P0, (size_t)b * nt * nt, LV, s_nleaf, s_pool);
        continue;
      }
      const long long off = s_pool;
      cd* UST = P0 + off;            // (U S)^T, r x m
      cd* VHT = UST + (size_t)r * m;  // (V^H)^T, n x r
      // UST[q][i] = sum_a Q[i][a] (A[a][perm q]), A = U S columns
      for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
        const int qq = e / m, i = e - (e / m) * m;
        const int pc = perm[qq];
        cd acc = make_double2(0, 0);
        for (int a = 0; a < k; ++a) acc = cfma(Y[(size_t)i * kPlrK + a], JA[a * k + pc], acc);
        UST[e] = acc;
      }
      // VHT[j][q] = conj(sum_a Q2[j][a] V[a][perm q])
      for (int e = threadIdx.x; e < r * n; e += blockDim.x) {
        const int j = e / r, qq = e - (e / r) * r;
        const int pc = perm[qq];
        cd acc = make_double2(0, 0);
        for (int a = 0; a < k; ++a) acc = cfma(Bt[(size_t)j * kPlrK + a], JV[a * k + pc], acc);
        VHT[e] = conjd(acc);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        LV[s_nleaf] = PlrLeaf{r0, c0, m, n, r, 1, (long long)b * nt * nt + off};  // absolute offset in the pool
        s_nleaf++;
        s_pool = off + (long long)r * (m + n);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) nleaves[b] = s_nleaf;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// application
// ---------------------------------------------------------------------------
// A projection task (PlrTask): leaf `leaf` of the block of term `term` of table row `row`.
// Arithmetic type of an apply: complex FP64 (double2) or complex FP32 (float2).
template <typename T>
struct Cx;
template <>
struct Cx<cd> {
  static __device__ __forceinline__ cd zero() { return make_double2(0, 0); }
  static __device__ __forceinline__ cd fma(cd a, cd b, cd c) { return cfma(a, b, c); }
  static __device__ __forceinline__ cd add(cd a, cd b) { return cadd(a, b); }
  static __device__ __forceinline__ cd from(cd v) { return v; }
  static __device__ __forceinline__ cd to_d(cd v) { return v; }
};
template <>
struct Cx<cf> {
  static __device__ __forceinline__ cf zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ cf fma(cf a, cf b, cf c) { return cfmaf(a, b, c); }
  static __device__ __forceinline__ cf add(cf a, cf b) { return make_float2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ cf from(cd v) { return make_float2((float)v.x, (float)v.y); }
  static __device__ __forceinline__ cd to_d(cf v) { return make_double2(v.x, v.y); }
};

constexpr int kProjWarps = 4;
constexpr int kExpWarps = 16;

// tbuf[s][task][q] = sign sum_j (V^H)^T[j][q] (x[in1] + x[in2])[c0 + j].
// One CTA per task: lane q, the kProjWarps warps split the columns j.
template <typename FT>
__global__ void __launch_bounds__(32 * kProjWarps) plr_project_kernel(
    int nt, int T4, const ApplyRow* __restrict__ table, const PlrTask* __restrict__ tasks, int ntasks,
    const PlrLeaf* __restrict__ leaves, const FT* __restrict__ pool, const cd* __restrict__ x, FT* __restrict__ tbuf,
    int rmax) {
  __shared__ FT part[kProjWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int task = blockIdx.x;
  const int s = blockIdx.y;
  const PlrTask tk = tasks[task];
  const ApplyTerm tm = table[tk.row].t[tk.term];
  const PlrLeaf lf = leaves[tk.leaf];
  const cd* xs = x + (size_t)s * T4 * nt;
  const cd* a = xs + (size_t)tm.in1 * nt + lf.c0;
  const cd* b2 = tm.in2 >= 0 ? xs + (size_t)tm.in2 * nt + lf.c0 : nullptr;
  const FT* VHT = pool + lf.off + (size_t)lf.rank * lf.m;
  FT acc = Cx<FT>::zero();
  if (lane < lf.rank) {
    for (int j = warp; j < lf.n; j += kProjWarps) {
      cd v = a[j];
      if (b2) v = cadd(v, b2[j]);
      acc = Cx<FT>::fma(VHT[(size_t)j * lf.rank + lane], Cx<FT>::from(cscale(v, tm.sign)), acc);
    }
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && lane < lf.rank) {
    FT v = part[0][lane];
#pragma unroll
    for (int w = 1; w < kProjWarps; ++w) v = Cx<FT>::add(v, part[w][lane]);
    tbuf[((size_t)s * ntasks + task) * rmax + lane] = v;
  }
}

// Per (row tile, table row, source): y[out][rows] = alpha (sum over terms and covering leaves + identity) + beta aux.
// tile_ptr/tile_leaf: CSR over (block, tile) of the leaves covering the tile; task_base[row*4+term] + lr_ord[leaf]
// is the projection task of a low-rank leaf.  Lane = row of the tile; warps take whole leaves.
template <typename FT>
__global__ void __launch_bounds__(32 * kExpWarps) plr_expand_kernel(
    int nt, int T4, const ApplyRow* __restrict__ table, const FT* __restrict__ pool,
    const PlrLeaf* __restrict__ leaves, const int* __restrict__ tile_ptr, const int* __restrict__ tile_leaf,
    int ntiles, const int* __restrict__ task_base, const int* __restrict__ lr_ord, const FT* __restrict__ tbuf,
    int ntasks, int rmax, const cd* x, const cd* __restrict__ aux, cd* y, double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FT* xin = reinterpret_cast<FT*>(smem_raw);  // 4 x nt
  __shared__ ApplyRow row;
  __shared__ FT part[kExpWarps][32];
  if (threadIdx.x == 0) row = table[blockIdx.y];
  __syncthreads();
  const int tile = blockIdx.x, s = blockIdx.z;
  const size_t vs = (size_t)T4 * nt;
  const cd* xs = x + s * vs;
  const cd* as = aux ? aux + s * vs : nullptr;
  for (int t = 0; t < row.nterms; ++t) {
    const ApplyTerm tm = row.t[t];
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      cd v = xs[(size_t)tm.in1 * nt + k];
      if (tm.in2 >= 0) v = cadd(v, xs[(size_t)tm.in2 * nt + k]);
      xin[t * nt + k] = Cx<FT>::from(cscale(v, tm.sign));
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = tile * 32 + lane;
  const FT* tb = tbuf + (size_t)s * ntasks * rmax;
  FT acc = Cx<FT>::zero();
  for (int t = 0; t < row.nterms; ++t) {
    const int blk = row.t[t].block;
    const int base = task_base[blockIdx.y * 4 + t];
    const FT* xv = xin + t * nt;
    const int e0 = tile_ptr[blk * ntiles + tile], e1 = tile_ptr[blk * ntiles + tile + 1];
    for (int e = e0 + warp; e < e1; e += kExpWarps) {
      const int li = tile_leaf[e];
      const PlrLeaf lf = leaves[li];
      const int i = r - lf.r0;
      if (i < 0 || i >= lf.m) continue;
      const FT* F = pool + lf.off;
      if (lf.kind == 0) {
        for (int j = 0; j < lf.n; ++j) acc = Cx<FT>::fma(F[(size_t)j * lf.m + i], xv[lf.c0 + j], acc);
      } else {
        const FT* tv = tb + (size_t)(base + lr_ord[li]) * rmax;
        for (int q = 0; q < lf.rank; ++q) acc = Cx<FT>::fma(F[(size_t)q * lf.m + i], tv[q], acc);
      }
    }
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && r < nt) {
    FT v = part[0][lane];
#pragma unroll
    for (int w = 1; w < kExpWarps; ++w) v = Cx<FT>::add(v, part[w][lane]);
    cd out = Cx<FT>::to_d(v);
    for (int e = 0; e < row.nid; ++e) {
      const cd* src = row.id_src[e] == 0 ? xs : as;
      out = cadd(out, cscale(src[(size_t)row.id_trace[e] * nt + r], row.id_sign[e]));
    }
    out = cscale(out, alpha);
    if (beta != 0.0) out = cadd(out, cscale(as[(size_t)row.out * nt + r], beta));
    y[s * vs + (size_t)row.out * nt + r] = out;
  }
}

__global__ void pool_to_fp32_kernel(const cd* __restrict__ src, cf* __restrict__ dst, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    cd v = src[q];
    dst[q] = make_float2((float)v.x, (float)v.y);
  }
}

// ---- launchers ----------------------------------------------------------------
size_t plr_scratch_per_cta(int nt) { return (size_t)4 * nt * kPlrK + (size_t)kPlrK * kPlrK; }
int plr_max_k() { return kPlrK; }

cudaError_t launch_plr_compress(int nt, const cd* blocks, const int* block_ids, int nblk, int rmax, double eps,
                                int oversample, cd* scratch, int nslots, PlrLeaf* leaves, int cap, int* nleaves,
                                cd* pool, int* status, cudaStream_t s) {
  const size_t smem = 2ull * kPlrK * kPlrK * sizeof(cd);
  cudaError_t e = smem_limit_max(reinterpret_cast<const void*>(plr_compress_kernel));
  if (e != cudaSuccess) return e;
  plr_compress_kernel<<<nslots, kPlrThreads, smem, s>>>(nt, blocks, block_ids, nblk, rmax, eps, oversample, scratch,
                                                        plr_scratch_per_cta(nt), leaves, cap, nleaves, pool, status);
  return cudaGetLastError();
}

cudaError_t launch_plr_apply(bool fp32, int nt, int T4, int /*ldd*/, const ApplyRow* table, int nrows,
                             const void* /*dense*/, const void* pool, const PlrLeaf* leaves, const PlrTask* tasks,
                             int ntasks, const int* tile_ptr, const int* tile_leaf, const int* task_base,
                             const int* lr_ord, cd* tbuf, int rmax, const cd* x, const cd* aux, cd* y, int nsrc,
                             double alpha, double beta, cudaStream_t s) {
  const int ntiles = (nt + 31) / 32;
  const size_t smem = 4ull * nt * (fp32 ? sizeof(cf) : sizeof(cd));
  if (ntasks > 0) {
    dim3 g1(ntasks, nsrc);
    if (fp32)
      plr_project_kernel<cf><<<g1, 32 * kProjWarps, 0, s>>>(nt, T4, table, tasks, ntasks, leaves, (const cf*)pool, x,
                                                            reinterpret_cast<cf*>(tbuf), rmax);
    else
      plr_project_kernel<cd><<<g1, 32 * kProjWarps, 0, s>>>(nt, T4, table, tasks, ntasks, leaves, (const cd*)pool, x,
                                                            tbuf, rmax);
  }
  dim3 g2(ntiles, nrows, nsrc);
  cudaError_t e;
  if (fp32) {
    e = smem_limit_max(reinterpret_cast<const void*>(plr_expand_kernel<cf>));
    plr_expand_kernel<cf><<<g2, 32 * kExpWarps, smem, s>>>(nt, T4, table, (const cf*)pool, leaves, tile_ptr,
                                                           tile_leaf, ntiles, task_base, lr_ord,
                                                           reinterpret_cast<const cf*>(tbuf), ntasks, rmax, x, aux, y,
                                                           alpha, beta);
  } else {
    e = smem_limit_max(reinterpret_cast<const void*>(plr_expand_kernel<cd>));
    plr_expand_kernel<cd><<<g2, 32 * kExpWarps, smem, s>>>(nt, T4, table, (const cd*)pool, leaves, tile_ptr,
                                                           tile_leaf, ntiles, task_base, lr_ord, tbuf, ntasks, rmax, x,
                                                           aux, y, alpha, beta);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_pool_to_fp32(const cd* src, cf* dst, size_t n, cudaStream_t s) {
  pool_to_fp32_kernel<<<1216, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace pt
