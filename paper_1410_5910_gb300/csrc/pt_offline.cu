// Offline phase (Algorithm 1) on the GPU, FP64.
//
//  * coef_kernel      the 5-point PML stencil of every local problem H^l
//                     (Section 2.1 discretization, Section 2.2 padding and
//                     normal extension), x-coupling coefficients W and E;
//  * factor_kernel    block elimination along x of the z-fastest local matrix:
//                     S_0 = D_0, S_i = D_i - diag(W_i) S_{i-1}^{-1} diag(E_{i-1}),
//                     each S_i inverted in shared memory by Gauss-Jordan with
//                     partial pivoting ("factorize local problems");
//  * extract_kernel   interface Green's matrices (Definition 1): solves with
//                     identity columns placed on the trace rows k in
//                     {0, 1, n, n+1}, read back on the trace rows j ("extract
//                     Green's functions"), stored as G(z_j, z_k)/h.
#include "pt_common.cuh"

namespace pt {

struct Stencil {
  cd center, north, south, west, east;
};

// Coefficients of row r (local array row) of grid column i of layer L's local
// problem: H u = center u + north u(r-1) + south u(r+1) + west u(i-1) + east u(i+1).
__device__ Stencil stencil(const Geometry& g, const LayerInfo& L, const double* __restrict__ c_ext, int i, int r) {
  int jr = r - L.pad_top;
  jr = jr < 0 ? 0 : (jr >= L.n ? L.n - 1 : jr);  // normal extension of m into the padding
  double c = c_ext[(size_t)(L.start + jr) * g.nt + i];
  double m = 1.0 / (c * c);
  double ih2 = 1.0 / (g.h * g.h);
  cd ax = pml_alpha(i, g.nt, g), axp = pml_alpha(i + 0.5, g.nt, g), axm = pml_alpha(i - 0.5, g.nt, g);
  cd az = pml_alpha(r, L.nloc, g), azp = pml_alpha(r + 0.5, L.nloc, g), azm = pml_alpha(r - 0.5, L.nloc, g);
  Stencil s;
  cd sx = cmul(ax, cadd(axp, axm));
  cd sz = cmul(az, cadd(azp, azm));
  s.center = make_double2((sx.x + sz.x) * ih2 - g.omega * g.omega * m, (sx.y + sz.y) * ih2);
  s.west = i > 0 ? cscale(cmul(ax, axm), -ih2) : make_double2(0, 0);
  s.east = i < g.nt - 1 ? cscale(cmul(ax, axp), -ih2) : make_double2(0, 0);
  s.north = r > 0 ? cscale(cmul(az, azm), -ih2) : make_double2(0, 0);
  s.south = r < L.nloc - 1 ? cscale(cmul(az, azp), -ih2) : make_double2(0, 0);
  return s;
}

__global__ void check_medium_kernel(const double* __restrict__ c_ext, size_t n, int* status) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double c = c_ext[k];
    if (!(c > 0.0) || !isfinite(c)) atomicOr(status, kErrNumeric);
  }
}

// grid (nt, L), block 128: W[l][i][r], E[l][i][r]
__global__ void coef_kernel(Geometry g, const LayerInfo* __restrict__ layers, const double* __restrict__ c_ext,
                            cd* __restrict__ W, cd* __restrict__ E) {
  const LayerInfo L = layers[blockIdx.y];
  int i = blockIdx.x;
  for (int r = threadIdx.x; r < L.nloc; r += blockDim.x) {
    Stencil s = stencil(g, L, c_ext, i, r);
    size_t o = L.coef_off + (size_t)i * L.nloc + r;
    W[o] = s.west;
    E[o] = s.east;
  }
}

// One CTA per layer.  Shared memory: A (nloc^2), colk (nloc), the stencil of
// the current column (centre, north, south, west) and the east couplings of
// the previous column (5 nloc), piv (nloc ints).
__global__ void __launch_bounds__(512) factor_kernel(Geometry g, const LayerInfo* __restrict__ layers,
                                                     const double* __restrict__ c_ext, cd* __restrict__ Sinv,
                                                     int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LayerInfo L = layers[blockIdx.x];
  const int n = L.nloc;
  cd* A = reinterpret_cast<cd*>(smem_raw);
  cd* colk = A + n * n;
  cd* s_cen = colk + n;
  cd* s_nor = s_cen + n;
  cd* s_sou = s_nor + n;
  cd* s_wes = s_sou + n;
  cd* s_eprev = s_wes + n;
  int* piv = reinterpret_cast<int*>(s_eprev + n);
  __shared__ int s_piv;
  __shared__ double s_pmax;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;

  for (int i = 0; i < g.nt; ++i) {
    // ---- S_i = D_i - diag(W_i) S_{i-1}^{-1} diag(E_{i-1}); A holds S_{i-1}^{-1} for i > 0
    for (int r = tid; r < n; r += nth) {
      Stencil st = stencil(g, L, c_ext, i, r);
      s_cen[r] = st.center; s_nor[r] = st.north; s_sou[r] = st.south; s_wes[r] = st.west;
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nth) {
      int r = idx / n, c = idx - r * n;
      cd v = make_double2(0, 0);
      if (i > 0) {
        v = cmul(cmul(s_wes[r], A[idx]), s_eprev[c]);
        v = make_double2(-v.x, -v.y);
      }
      if (c == r) v = cadd(v, s_cen[r]);
      else if (c == r - 1) v = cadd(v, s_nor[r]);
      else if (c == r + 1) v = cadd(v, s_sou[r]);
      A[idx] = v;
    }
    __syncthreads();
    // east couplings of this column, used when forming S_{i+1}
    for (int r = tid; r < n; r += nth) s_eprev[r] = stencil(g, L, c_ext, i, r).east;
    // ---- in-place Gauss-Jordan inversion with partial (row) pivoting
    for (int k = 0; k < n; ++k) {
      if (warp == 0) {
        double best = -1.0;
        int bi = k;
        for (int r = k + lane; r < n; r += 32) {
          double v = cabs2(A[r * n + k]);
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          double ob = __shfl_down_sync(0xffffffffu, best, o);
          int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_piv = bi; s_pmax = best; piv[k] = bi; }
      }
      __syncthreads();
      const int p = s_piv;
      if (s_pmax <= 0.0 || !isfinite(s_pmax)) {
        if (tid == 0) atomicOr(status, kErrSingular);
        // keep going on a unit pivot so that the kernel ends normally
        if (tid == 0) A[k * n + k] = make_double2(1.0, 0.0);
        __syncthreads();
      } else if (p != k) {
        for (int c = tid; c < n; c += nth) {
          cd t = A[k * n + c];
          A[k * n + c] = A[p * n + c];
          A[p * n + c] = t;
        }
        __syncthreads();
      }
      const cd d = cinv(A[k * n + k]);
      for (int r = tid; r < n; r += nth) colk[r] = A[r * n + k];
      __syncthreads();
      for (int c = tid; c < n; c += nth) A[k * n + c] = (c == k) ? d : cmul(A[k * n + c], d);
      __syncthreads();
      for (int r = warp; r < n; r += nth / 32) {
        if (r == k) continue;
        const cd t = colk[r];
        for (int c = lane; c < n; c += 32) {
          cd a = (c == k) ? make_double2(0, 0) : A[r * n + c];
          cd b = A[k * n + c];
          A[r * n + c] = make_double2(a.x - (t.x * b.x - t.y * b.y), a.y - (t.x * b.y + t.y * b.x));
        }
      }
      __syncthreads();
    }
    // undo the row pivoting: swap columns in reverse order
    for (int k = n - 1; k >= 0; --k) {
      int p = piv[k];
      if (p != k) {
        for (int r = tid; r < n; r += nth) {
          cd t = A[r * n + k];
          A[r * n + k] = A[r * n + p];
          A[r * n + p] = t;
        }
      }
      __syncthreads();
    }
    cd* dst = Sinv + L.sinv_off + (size_t)i * n * n;
    for (int idx = tid; idx < n * n; idx += nth) dst[idx] = A[idx];
    __syncthreads();
  }
}

// Persistent: CTA b handles tasks b, b + gridDim.x, ...  Shared memory:
// two nloc x 32 complex buffers.  Yslot: per-CTA scratch of nt * nloc_max * 32.
__global__ void __launch_bounds__(256) extract_kernel(Geometry g, const LayerInfo* __restrict__ layers,
                                                      const ExtractTask* __restrict__ tasks, int ntasks,
                                                      const cd* __restrict__ Sinv, const cd* __restrict__ W,
                                                      const cd* __restrict__ E, cd* __restrict__ Yscratch,
                                                      size_t slot_elems, cd* __restrict__ blocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = 32;
  constexpr int RPW = (kMaxNloc + 7) / 8;  // rows per warp (8 warps)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cd* Y = Yscratch + (size_t)blockIdx.x * slot_elems;
  const double ih2 = 1.0 / (g.h * g.h);
  const size_t nt = g.nt, bsz = nt * nt;

  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const ExtractTask T = tasks[t];
    const LayerInfo L = layers[T.layer];
    const int n = L.nloc;
    cd* vbuf = reinterpret_cast<cd*>(smem_raw);  // n x R
    cd* ybuf = vbuf + n * R;                      // n x R
    // the RHS column q = a * w_count + b : source row kk index a, source column c0 + b
    const int q = lane;
    const int qa = q / T.w, qb = q - (q / T.w) * T.w;
    const bool qvalid = (qa < T.nk) && (T.c0 + qb < g.nt);
    const int qrow = qvalid ? L.row[T.kk[qa]] : -1;
    const int qcol = T.c0 + qb;

    for (int r = threadIdx.x; r < n * R; r += blockDim.x) ybuf[r] = make_double2(0, 0);
    __syncthreads();
    // ---------------- forward: y_i = Sinv_i (F_i - W_i o y_{i-1}) for i >= c0
    for (int i = T.c0; i < g.nt; ++i) {
      const cd* Wi = W + L.coef_off + (size_t)i * n;
      for (int r = warp; r < n; r += 8) {
        cd yp = ybuf[r * R + q];
        cd v = cmul(Wi[r], yp);
        v = make_double2(-v.x, -v.y);
        if (qvalid && i == qcol && r == qrow) v.x += 1.0;
        vbuf[r * R + q] = v;
      }
      __syncthreads();
      const cd* S = Sinv + L.sinv_off + (size_t)i * n * n;
      cd acc[RPW];
#pragma unroll
      for (int a = 0; a < RPW; ++a) acc[a] = make_double2(0, 0);
      for (int kk = 0; kk < n; ++kk) {
        cd b = vbuf[kk * R + q];
#pragma unroll
        for (int a = 0; a < RPW; ++a) {
          int r = warp + 8 * a;
          if (r < n) acc[a] = cfma(__ldg(S + (size_t)r * n + kk), b, acc[a]);
        }
      }
      cd* Yi = Y + (size_t)i * n * R;
#pragma unroll
      for (int a = 0; a < RPW; ++a) {
        int r = warp + 8 * a;
        if (r < n) { ybuf[r * R + q] = acc[a]; Yi[r * R + q] = acc[a]; }
      }
      __syncthreads();
    }
    // ---------------- backward: x_i = y_i - Sinv_i (E_i o x_{i+1}); ybuf holds x_{i+1}
    for (int i = g.nt - 1; i >= 0; --i) {
      if (i < g.nt - 1) {
        const cd* Ei = E + L.coef_off + (size_t)i * n;
        for (int r = warp; r < n; r += 8) vbuf[r * R + q] = cmul(Ei[r], ybuf[r * R + q]);
        __syncthreads();
        const cd* S = Sinv + L.sinv_off + (size_t)i * n * n;
        cd acc[RPW];
#pragma unroll
        for (int a = 0; a < RPW; ++a) acc[a] = make_double2(0, 0);
        for (int kk = 0; kk < n; ++kk) {
          cd b = vbuf[kk * R + q];
#pragma unroll
          for (int a = 0; a < RPW; ++a) {
            int r = warp + 8 * a;
            if (r < n) acc[a] = cfma(__ldg(S + (size_t)r * n + kk), b, acc[a]);
          }
        }
        const cd* Yi = Y + (size_t)i * n * R;
#pragma unroll
        for (int a = 0; a < RPW; ++a) {
          int r = warp + 8 * a;
          if (r < n) {
            cd y = (i >= T.c0) ? Yi[r * R + q] : make_double2(0, 0);
            ybuf[r * R + q] = csub(y, acc[a]);
          }
        }
        __syncthreads();
      }
      // x_i (in ybuf) at the target rows -> blocks
      if (qvalid) {
        for (int jj = warp; jj < 4; jj += 8) {
          int rj = L.row[jj];
          if (rj < 0) continue;
          cd v = cscale(ybuf[rj * R + q], ih2);
          blocks[((size_t)T.layer * 16 + jj * 4 + T.kk[qa]) * bsz + (size_t)i * nt + qcol] = v;
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
cudaError_t launch_check_medium(const double* c, size_t n, int* status, cudaStream_t s) {
  check_medium_kernel<<<304, 256, 0, s>>>(c, n, status);
  return cudaGetLastError();
}

cudaError_t launch_coef(const Geometry& g, const LayerInfo* layers, const double* c, cd* W, cd* E, cudaStream_t s) {
  coef_kernel<<<dim3(g.nt, g.L), 128, 0, s>>>(g, layers, c, W, E);
  return cudaGetLastError();
}

cudaError_t launch_factor(const Geometry& g, const LayerInfo* layers, int nloc_max, const double* c, cd* Sinv,
                          int* status, cudaStream_t s) {
  size_t smem = (size_t)nloc_max * nloc_max * sizeof(cd) + 6ull * nloc_max * sizeof(cd) + nloc_max * sizeof(int);
  cudaError_t e = smem_limit_max(reinterpret_cast<const void*>(factor_kernel));
  if (e != cudaSuccess) return e;
  factor_kernel<<<g.L, 512, smem, s>>>(g, layers, c, Sinv, status);
  return cudaGetLastError();
}

cudaError_t launch_extract(const Geometry& g, const LayerInfo* layers, const ExtractTask* tasks, int ntasks,
                           int nslots, int nloc_max, const cd* Sinv, const cd* W, const cd* E, cd* Y,
                           size_t slot_elems, cd* blocks, cudaStream_t s) {
  size_t smem = 2ull * nloc_max * 32 * sizeof(cd);
  cudaError_t e = smem_limit_max(reinterpret_cast<const void*>(extract_kernel));
  if (e != cudaSuccess) return e;
  extract_kernel<<<nslots, 256, smem, s>>>(g, layers, tasks, ntasks, Sinv, W, E, Y, slot_elems, blocks);
  return cudaGetLastError();
}


}  // namespace pt
