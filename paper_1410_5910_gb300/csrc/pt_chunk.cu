// Local solves split along x into K chunks per layer.
//
// The substitutions of the block factorization (Section 2.2, Algorithm 1)
//   forward  y_i = Sinv_i (f_i - W_i o y_{i-1}),   backward x_i = y_i - Sinv_i (E_i o x_{i+1})
// are affine recurrences in the column index i, so they can be cut into chunks of
// columns [a_k, b_k] (an exact reorganisation, not in the paper).  With
// A_i = -Sinv_i diag(W_i) and B_i = -Sinv_i diag(E_i), and y', x'' the chunk's
// solution from zero boundary values,
//   y_i     = y'_i + Phi_i beta_k,                 Phi_i = A_i ... A_{a_k},  beta_k = y_{a_k - 1},
//   x_{a_k} = x''_{a_k} + M_k beta_k + Psi_k gamma_k,                       gamma_k = x_{b_k + 1},
//   M_k = sum_{j = a_k}^{b_k} (B_{a_k} ... B_{j-1}) Phi_j,   Psi_k = B_{a_k} ... B_{b_k}.
// An online local solve is then (1) every chunk from zero boundaries, all in parallel,
// keeping y'_{b_k} and x''_{a_k}; (2) per layer, beta_{k+1} = y'_{b_k} + Phi_k beta_k
// (Phi_k = Phi_{b_k}) and gamma_{k-1} = x''_{a_k} + M_k beta_k + Psi_k gamma_k; (3) every
// chunk again from beta_k and gamma_k, emitting its traces or its part of the volume.
// The dependent chain is 2 (b_k - a_k + 1) column steps plus 2 K small products instead
// of 2 n_t - 1 column steps.  Phi_k, M_k, Psi_k are formed offline in FP64 and kept in
// complex64; the online arithmetic is that of the FP32 local solves (Sinv_i rounded to
// complex64).
#include "pt_common.cuh"

#include <algorithm>

namespace pt {

// ---- offline: Phi_k, M_k, Psi_k of every (layer, chunk), FP64 -----------------------
// One CTA per (chunk, layer) runs the chunk's columns in order, with
//   Phi <- A_j Phi,  M <- M + G Phi,  G <- G B_j     (Phi = G = I, M = 0 at the start),
// so that at the end Phi = Phi_{b_k}, M = M_k, G = Psi_k.  The n x n working matrices
// live in global scratch (L2); every product is n^3 complex multiply-adds on the FP64
// pipe.  W_0 and E_{n_t - 1} couple to columns outside the grid and count as zero.
constexpr int kChunkGemmThreads = 256;

__device__ __forceinline__ int chunk_lo(int k, int nt, int K) { return (int)(((long long)k * nt) / K); }

// C = alpha A B (+ C when acc); n x n row-major, C distinct from A and B
__device__ void chunk_gemm(const cd* A, const cd* B, cd* C, int n, double alpha, bool acc) {
  const int nn = n * n;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    const cd* a = A + (size_t)r * n;
    double sr = 0.0, si = 0.0, tr = 0.0, ti = 0.0;
    int k = 0;
    for (; k + 1 < n; k += 2) {
      const cd a0 = a[k], a1 = a[k + 1];
      const cd b0 = B[(size_t)k * n + c], b1 = B[(size_t)(k + 1) * n + c];
      sr = fma(a0.x, b0.x, sr);
      sr = fma(-a0.y, b0.y, sr);
      si = fma(a0.x, b0.y, si);
      si = fma(a0.y, b0.x, si);
      tr = fma(a1.x, b1.x, tr);
      tr = fma(-a1.y, b1.y, tr);
      ti = fma(a1.x, b1.y, ti);
      ti = fma(a1.y, b1.x, ti);
    }
    if (k < n) {
      const cd a0 = a[k], b0 = B[(size_t)k * n + c];
      sr = fma(a0.x, b0.x, sr);
      sr = fma(-a0.y, b0.y, sr);
      si = fma(a0.x, b0.y, si);
      si = fma(a0.y, b0.x, si);
    }
    cd v = make_double2(alpha * (sr + tr), alpha * (si + ti));
    if (acc) v = cadd(C[e], v);
    C[e] = v;
  }
}

__global__ void __launch_bounds__(kChunkGemmThreads)
    chunk_transfer_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cd* __restrict__ Sinv,
                          const cd* __restrict__ Wc, const cd* __restrict__ Ec, int K, int nmax, cd* work,
                          cf* __restrict__ out) {
  const int k = blockIdx.x, l = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt, nn = n * n;
  const size_t slot = (size_t)nmax * nmax;
  cd* Phi = work + ((size_t)l * K + k) * 4 * slot;
  cd* M = Phi + slot;
  cd* G = M + slot;
  cd* T = G + slot;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    const cd one = make_double2(r == c ? 1.0 : 0.0, 0.0);
    Phi[e] = one;
    G[e] = one;
    M[e] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int a = chunk_lo(k, nt, K), b = chunk_lo(k + 1, nt, K) - 1;
  for (int j = a; j <= b; ++j) {
    const cd* S = Sinv + L.sinv_off + (size_t)j * nn;
    const cd* w = Wc + L.coef_off + (size_t)j * n;
    const cd* ec = Ec + L.coef_off + (size_t)j * n;
    // T = W_j o_rows Phi
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int r = e / n;
      T[e] = j > 0 ? cmul(__ldg(w + r), Phi[e]) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    chunk_gemm(S, T, Phi, n, -1.0, false);  // Phi = A_j Phi
    __syncthreads();
    chunk_gemm(G, Phi, M, n, 1.0, true);    // M += G Phi
    chunk_gemm(G, S, T, n, 1.0, false);     // T = G Sinv_j
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {  // G = G B_j = -T o_cols E_j
      const int c = e % n;
      G[e] = j < nt - 1 ? cscale(cmul(T[e], __ldg(ec + c)), -1.0) : make_double2(0.0, 0.0);
    }
    __syncthreads();
  }
  cf* o = out + ((size_t)l * K + k) * 3 * slot;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    o[e] = make_float2((float)Phi[e].x, (float)Phi[e].y);
    o[slot + e] = make_float2((float)M[e].x, (float)M[e].y);
    o[2 * slot + e] = make_float2((float)G[e].x, (float)G[e].y);
  }
}

size_t chunk_work_bytes(int L, int K, int nmax) { return (size_t)L * K * 4 * nmax * nmax * sizeof(cd); }

cudaError_t launch_chunk_transfer(const Geometry& g, const LayerInfo* layers, const cd* Sinv, const cd* W,
                                  const cd* E, int K, int nmax, cd* work, cf* out, cudaStream_t s) {
  chunk_transfer_kernel<<<dim3(K, g.L), kChunkGemmThreads, 0, s>>>(g, layers, Sinv, W, E, K, nmax, work, out);
  return cudaGetLastError();
}

// ---- online: one chunk of one layer for one source, one CTA -------------------------
// The arithmetic of the single-CTA FP32 local solve: Sinv_i (complex64) by one bulk
// asynchronous copy per column into a double buffer (mbarrier, bounded wait), four
// threads per row.  PHASE 1 starts both substitutions from zero and keeps y'_{b_k}
// and x''_{a_k} (bnd slots 0 and 1); PHASE 3 starts from beta_k, gamma_k (slots 2, 3)
// and emits: MODE 0 the chunk's part of the right-hand side traces, MODE 1 its columns
// of the volume (complex64; converted to FP64 by a separate pass).  The source and the
// trace forcing arrive in complex64 as well (converted once per solve): no FP64
// instruction, which holds the SM's FP64 pipe for 16 cycles per warp on GB300, is left
// in the column steps.
constexpr int kChunkThreads = 512;
constexpr int kChunkQ = 4;  // threads per row

__device__ __forceinline__ uint32_t chunk_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long chunk_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool chunk_mb_wait(uint64_t* bar, int parity, int* status) {
  const unsigned long long t0 = chunk_timer();
  for (long long it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(chunk_saddr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && chunk_timer() - t0 > 2000000000ull) break;
  }
  atomicOr(status, kErrTimeout);
  return false;
}
// a Sinv buffer: nloc_max^2 complex64 plus one slack element in front (a block that starts
// 8 bytes off a 16-byte boundary) and one behind, rounded to an even count
__host__ __device__ inline size_t chunk_buf_elems(int nmax) { return ((size_t)nmax * nmax + 3) & ~(size_t)1; }
size_t chunk_solve_smem(int nmax) { return (2 * chunk_buf_elems(nmax) + (size_t)kMaxNloc) * sizeof(cf); }

template <int MODE, int PHASE>
__global__ void __launch_bounds__(kChunkThreads, 1)
    layer_solve_chunk_kernel(Geometry g, const LayerInfo* __restrict__ layers, int K, const cf* __restrict__ Shi,
                             const cf* __restrict__ Whi, const cf* __restrict__ Ehi, const cf* __restrict__ f,
                             const cf* __restrict__ xtr, cf* __restrict__ Ystore, size_t ystride,
                             cd* __restrict__ out, cf* __restrict__ vol, const int* __restrict__ nzflag, int nmax,
                             cf* __restrict__ bnd,
                             int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  const int l = blockIdx.x / K, kc = blockIdx.x - l * K, s = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt;
  const int T = 2 * (g.L - 1);
  const size_t T4n = (size_t)2 * T * nt;
  const int a = chunk_lo(kc, nt, K), b = chunk_lo(kc + 1, nt, K) - 1, len = b - a + 1;
  cf* bk = bnd + (((size_t)s * g.L + l) * K + kc) * 4 * nmax;
  const size_t bufel = chunk_buf_elems(nmax);
  cf* B0 = reinterpret_cast<cf*>(smem);
  cf* B1 = B0 + bufel;
  cf* vloc = B1 + bufel;  // [kMaxNloc]
  const bool fnz = nzflag[s * g.L + l] != 0;

  if (MODE == 0 && !fnz) {  // no source in this layer: its traces are zero (phase 2 skips it too)
    if (PHASE == 3) {
      cd* o = out + (size_t)s * T4n;
      for (int i = a + threadIdx.x; i <= b; i += blockDim.x) {
        if (L.has_bot) {
          o[(size_t)(2 * l) * nt + i] = make_double2(0, 0);
          o[(size_t)(2 * l + 1) * nt + i] = make_double2(0, 0);
        }
        if (L.has_top) {
          o[(size_t)(T + 2 * (l - 1)) * nt + i] = make_double2(0, 0);
          o[(size_t)(T + 2 * (l - 1) + 1) * nt + i] = make_double2(0, 0);
        }
      }
    }
    return;
  }

  const int r = threadIdx.x / kChunkQ, q = threadIdx.x % kChunkQ;
  const bool own = r < n && q == 0;  // owner of row r's chain state
  const int per = (n + kChunkQ - 1) / kChunkQ;
  const int k0 = q * per, k1 = min(n, k0 + per);
  const cf* fs = f + (size_t)s * g.Nz * nt;
  const cf* xs = (MODE == 1) ? xtr + (size_t)s * T4n : nullptr;
  cf* Y = Ystore + ((size_t)s * g.L + l) * ystride;
  const int nsteps = 2 * len;
  auto col = [&](int st) { return st < len ? a + st : b - (st - len); };
  const bool in_layer = own && r >= L.pad_top && r < L.pad_top + L.n;
  const size_t frow = in_layer ? (size_t)(L.start + r - L.pad_top) * nt : 0;
  int ftr = -1;
  float fsg = 0.f;
  if (MODE == 1 && own) {
    const float ih2 = (float)(1.0 / (g.h * g.h));
    if (L.has_top && r == L.row[1]) { ftr = 2 * (l - 1); fsg = ih2; }
    if (L.has_top && r == L.row[0]) { ftr = 2 * (l - 1) + 1; fsg = -ih2; }
    if (L.has_bot && r == L.row[3]) { ftr = 2 * l; fsg = -ih2; }
    if (L.has_bot && r == L.row[2]) { ftr = 2 * l + 1; fsg = ih2; }
  }
  int emit = -1;  // MODE 0: output trace of this row
  if (MODE == 0 && own) {
    if (L.has_bot && r == L.row[2]) emit = 2 * l;
    if (L.has_bot && r == L.row[3]) emit = 2 * l + 1;
    if (L.has_top && r == L.row[0]) emit = T + 2 * (l - 1);
    if (L.has_top && r == L.row[1]) emit = T + 2 * (l - 1) + 1;
  }
  const int nn = n * n;
  auto src_of = [&](int st) { return Shi + L.sinv_off + (size_t)col(st) * nn; };
  auto view_of = [&](int st) {
    cf* B = (st & 1) ? B1 : B0;
    return ((reinterpret_cast<uintptr_t>(src_of(st)) & 15) != 0) ? B + 1 : B;
  };

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(chunk_saddr(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(chunk_saddr(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // one thread: the 16-byte aligned bulk part by the copy engine, an odd head / tail by hand
  auto stage = [&](int st) {
    if (threadIdx.x != 0) return;
    const cf* src = src_of(st);
    cf* view = view_of(st);
    const int head = (reinterpret_cast<uintptr_t>(src) & 15) ? 1 : 0;
    const int m = nn - head;
    const int nbulk = m & ~1;
    if (head) view[0] = src[0];
    if (m & 1) view[nn - 1] = src[nn - 1];
    uint64_t* bb = &bar[st & 1];
    const uint32_t bytes = (uint32_t)nbulk * (uint32_t)sizeof(cf);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic reads of the buffer first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(chunk_saddr(bb)), "r"(bytes)
                 : "memory");
    if (nbulk > 0)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              chunk_saddr(view + head)),
          "l"(src + head), "r"(bytes), "r"(chunk_saddr(bb))
          : "memory");
  };
  // per-row operands of a step, prefetched one step ahead by the row owner
  cf c_next = make_float2(0.f, 0.f), y_next = make_float2(0.f, 0.f);
  cf f_next = make_float2(0.f, 0.f), ta_next = make_float2(0.f, 0.f), tb_next = make_float2(0.f, 0.f);
  auto prefetch = [&](int st) {
    if (!own) return;
    const int i = col(st);
    const bool fwd = st < len;
    // W_0 and E_{n_t - 1} couple to columns outside the grid
    const bool edge = fwd ? i == 0 : i == nt - 1;
    c_next = edge ? make_float2(0.f, 0.f) : __ldg((fwd ? Whi : Ehi) + L.coef_off + (size_t)i * n + r);
    if (fwd) {
      cf v = make_float2(0.f, 0.f);
      if (fnz && in_layer) v = fs[frow + i];
      f_next = v;
      if (MODE == 1 && ftr >= 0) {
        ta_next = xs[(size_t)ftr * nt + i];
        tb_next = xs[(size_t)(T + ftr) * nt + i];
      }
    } else {
      y_next = Y[(size_t)i * n + r];
    }
  };

  // y_{i-1} (forward) / x_{i+1} (backward) of row r: beta_k, later gamma_k, in phase 3
  cf chain = make_float2(0.f, 0.f);
  if (PHASE == 3 && own) chain = bk[2 * nmax + r];
  stage(0);
  prefetch(0);
  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < len;
    const int i = col(st);
    cf yst = y_next;
    if (st == len && own) {  // the forward substitution is done: y_{b_k} -> x_{b_k + 1}
      yst = chain;           // y_{b_k} (its stored copy is written in this step's predecessor)
      if (PHASE == 1) bk[r] = chain;
      chain = PHASE == 3 ? bk[3 * nmax + r] : make_float2(0.f, 0.f);
    }
    const cf c = c_next;
    const cf fv = f_next, ta = ta_next, tb = tb_next;
    if (st + 1 < nsteps) prefetch(st + 1);
    // (a) right-hand side of row r
    if (own) {
      float vr, vi;
      if (fwd) {
        float dr = fv.x, di = fv.y;
        if (MODE == 1 && ftr >= 0) {
          dr = fmaf(fsg, ta.x + tb.x, dr);
          di = fmaf(fsg, ta.y + tb.y, di);
        }
        vr = dr - (c.x * chain.x - c.y * chain.y);
        vi = di - (c.x * chain.y + c.y * chain.x);
      } else {
        vr = c.x * chain.x - c.y * chain.y;
        vi = c.x * chain.y + c.y * chain.x;
      }
      vloc[r] = make_float2(vr, vi);
    }
    // Sinv_i in shared memory: phase (st / 2) of the buffer's barrier (bounded wait)
    if (!chunk_mb_wait(&bar[st & 1], (st >> 1) & 1, status)) return;
    __syncthreads();  // vloc, the hand-copied elements and Sinv_i visible to all
    if (st + 1 < nsteps) stage(st + 1);  // the other buffer was last read in step st - 1
    // (b) row r of Sinv_i v, a quarter of the columns per thread
    const cf* Srow = view_of(st) + (size_t)min(r, n - 1) * n;
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      const cf a0 = Srow[k], a1 = Srow[k + 1];
      const cf v0 = vloc[k], v1 = vloc[k + 1];
      ar = fmaf(a0.x, v0.x, ar); ar = fmaf(-a0.y, v0.y, ar);
      ai = fmaf(a0.x, v0.y, ai); ai = fmaf(a0.y, v0.x, ai);
      br = fmaf(a1.x, v1.x, br); br = fmaf(-a1.y, v1.y, br);
      bi = fmaf(a1.x, v1.y, bi); bi = fmaf(a1.y, v1.x, bi);
    }
    if (k < k1) {
      const cf a0 = Srow[k], v0 = vloc[k];
      ar = fmaf(a0.x, v0.x, ar); ar = fmaf(-a0.y, v0.y, ar);
      ai = fmaf(a0.x, v0.y, ai); ai = fmaf(a0.y, v0.x, ai);
    }
    ar += br;
    ai += bi;
    ar += __shfl_xor_sync(0xffffffffu, ar, 1);
    ai += __shfl_xor_sync(0xffffffffu, ai, 1);
    ar += __shfl_xor_sync(0xffffffffu, ar, 2);
    ai += __shfl_xor_sync(0xffffffffu, ai, 2);
    if (own) {
      if (fwd) {
        chain = make_float2(ar, ai);
        Y[(size_t)i * n + r] = chain;
      } else {
        chain = make_float2(yst.x - ar, yst.y - ai);
        if (PHASE == 3) {
          if (MODE == 0) {
            if (emit >= 0)
              out[(size_t)s * T4n + (size_t)emit * nt + i] = make_double2(-(double)chain.x, -(double)chain.y);
          } else if (in_layer) {
            vol[(size_t)s * g.Nz * nt + frow + i] = chain;
          }
        }
      }
    }
    __syncthreads();  // vloc is rewritten in the next step
  }
  if (PHASE == 1 && own) bk[nmax + r] = chain;  // x''_{a_k}
}

// ---- phase 2: the chunk boundary values of each (layer, source) ---------------------
// beta_0 = 0, beta_{k+1} = y'_{b_k} + Phi_k beta_k;  gamma_{K-1} = 0,
// gamma_{k-1} = x''_{a_k} + M_k beta_k + Psi_k gamma_k.  Warp w owns rows w + 16 j
// (j < 8); lane (rg, cg) = (lane / 8, lane % 8) takes rows j = rg, rg + 4 and the columns
// cg + 8 u, so eight lanes read 64 contiguous bytes of a row, a product is one round trip
// (every load of the lane in flight), and a row sum needs three shuffles.  The vector is
// held in registers; the betas and the phase-1 boundary values stay in shared memory;
// every matrix of the layer is requested into L2 when the CTA starts.
constexpr int kPropThreads = 512;
constexpr int kPropWarps = kPropThreads / 32;
constexpr int kPropCols = (kMaxNloc + 7) / 8;  // columns per lane

__global__ void __launch_bounds__(kPropThreads)
    chunk_propagate_kernel(Geometry g, const LayerInfo* __restrict__ layers, int K, int nmax,
                           const cf* __restrict__ Tm, const int* __restrict__ nzflag, int mode, cf* __restrict__ bnd) {
  static_assert(kPropWarps * 8 >= kMaxNloc, "eight rows per warp cover a local problem");
  extern __shared__ __align__(16) unsigned char smem[];
  const int l = blockIdx.x, s = blockIdx.y;
  const int n = layers[l].nloc;
  if (mode == 0 && nzflag[s * g.L + l] == 0) return;
  cf* beta = reinterpret_cast<cf*>(smem);  // [K][nmax]
  cf* gam = beta + (size_t)K * nmax;       // [nmax]
  cf* yb = gam + nmax;                     // [K][nmax]: y'_{b_k}
  cf* xa = yb + (size_t)K * nmax;          // [K][nmax]: x''_{a_k}
  const size_t slot = (size_t)nmax * nmax;
  cf* bl = bnd + ((size_t)s * g.L + l) * K * 4 * nmax;
  const cf* Tl = Tm + (size_t)l * K * 3 * slot;
  for (int i = threadIdx.x; i < K * n; i += blockDim.x) {  // the phase-1 boundary values, off the chain
    const int k = i / n, r = i - k * n;
    yb[(size_t)k * nmax + r] = bl[((size_t)k * 4 + 0) * nmax + r];
    xa[(size_t)k * nmax + r] = bl[((size_t)k * 4 + 1) * nmax + r];
  }
  for (int i = threadIdx.x; i < 3 * K; i += blockDim.x) {  // L2 prefetch hints, 16-byte aligned parts
    const uintptr_t p0 = reinterpret_cast<uintptr_t>(Tl + (size_t)i * slot);
    const uintptr_t a0 = (p0 + 15) & ~(uintptr_t)15, a1 = (p0 + (size_t)n * n * sizeof(cf)) & ~(uintptr_t)15;
    if (a1 > a0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rg = lane >> 3, cg = lane & 7;
  const int row0 = warp + kPropWarps * rg, row1 = warp + kPropWarps * (rg + 4);
  for (int i = threadIdx.x; i < nmax; i += blockDim.x) {
    beta[i] = make_float2(0.f, 0.f);
    gam[i] = make_float2(0.f, 0.f);
    bl[2 * nmax + i] = make_float2(0.f, 0.f);                          // beta_0
    bl[((size_t)(K - 1) * 4 + 3) * nmax + i] = make_float2(0.f, 0.f);  // gamma_{K-1}
  }
  __syncthreads();
  // acc0 / acc1 += rows row0 / row1 of A times v, summed over the eight lanes of the row group
  auto gemv = [&](const cf* A, const cf* v, float2& acc0, float2& acc1) {
    cf xr[kPropCols], m0[kPropCols], m1[kPropCols];
#pragma unroll
    for (int u = 0; u < kPropCols; ++u) {
      const int col = cg + 8 * u;
      xr[u] = col < n ? v[col] : make_float2(0.f, 0.f);
      m0[u] = (row0 < n && col < n) ? __ldg(A + (size_t)row0 * n + col) : make_float2(0.f, 0.f);
      m1[u] = (row1 < n && col < n) ? __ldg(A + (size_t)row1 * n + col) : make_float2(0.f, 0.f);
    }
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
    for (int u = 0; u < kPropCols; ++u) {
      ar = fmaf(m0[u].x, xr[u].x, ar);
      ar = fmaf(-m0[u].y, xr[u].y, ar);
      ai = fmaf(m0[u].x, xr[u].y, ai);
      ai = fmaf(m0[u].y, xr[u].x, ai);
      br = fmaf(m1[u].x, xr[u].x, br);
      br = fmaf(-m1[u].y, xr[u].y, br);
      bi = fmaf(m1[u].x, xr[u].y, bi);
      bi = fmaf(m1[u].y, xr[u].x, bi);
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
      br += __shfl_xor_sync(0xffffffffu, br, o);
      bi += __shfl_xor_sync(0xffffffffu, bi, o);
    }
    acc0.x += ar;
    acc0.y += ai;
    acc1.x += br;
    acc1.y += bi;
  };
  for (int k = 0; k + 1 < K; ++k) {
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    gemv(Tl + (size_t)k * 3 * slot, beta + (size_t)k * nmax, a0, a1);
    if (cg == 0) {
      if (row0 < n) {
        const cf y = yb[(size_t)k * nmax + row0];
        const cf v = make_float2(y.x + a0.x, y.y + a0.y);
        beta[(size_t)(k + 1) * nmax + row0] = v;
        bl[((size_t)(k + 1) * 4 + 2) * nmax + row0] = v;
      }
      if (row1 < n) {
        const cf y = yb[(size_t)k * nmax + row1];
        const cf v = make_float2(y.x + a1.x, y.y + a1.y);
        beta[(size_t)(k + 1) * nmax + row1] = v;
        bl[((size_t)(k + 1) * 4 + 2) * nmax + row1] = v;
      }
    }
    __syncthreads();
  }
  for (int k = K - 1; k >= 1; --k) {
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    gemv(Tl + ((size_t)k * 3 + 1) * slot, beta + (size_t)k * nmax, a0, a1);
    asm volatile("" ::: "memory");  // one matrix's loads in flight at a time (registers)
    gemv(Tl + ((size_t)k * 3 + 2) * slot, gam, a0, a1);
    __syncthreads();  // every warp has read gamma_k
    if (cg == 0) {
      if (row0 < n) {
        const cf x = xa[(size_t)k * nmax + row0];
        const cf v = make_float2(x.x + a0.x, x.y + a0.y);
        gam[row0] = v;
        bl[((size_t)(k - 1) * 4 + 3) * nmax + row0] = v;
      }
      if (row1 < n) {
        const cf x = xa[(size_t)k * nmax + row1];
        const cf v = make_float2(x.x + a1.x, x.y + a1.y);
        gam[row1] = v;
        bl[((size_t)(k - 1) * 4 + 3) * nmax + row1] = v;
      }
    }
    __syncthreads();
  }
}

// complex64 copies of FP64 data for the column steps, and the FP64 volume from its
// complex64 result: elementwise, spread over every SM
__global__ void to_c64_kernel(const cd* __restrict__ a, size_t n, cf* __restrict__ b) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const cd v = a[k];
    b[k] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void to_c128_kernel(const cf* __restrict__ a, size_t n, cd* __restrict__ b) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const cf v = a[k];
    b[k] = make_double2((double)v.x, (double)v.y);
  }
}
cudaError_t launch_to_c64(const cd* a, size_t n, cf* b, cudaStream_t s) {
  const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
  to_c64_kernel<<<grid, 256, 0, s>>>(a, n, b);
  return cudaGetLastError();
}

// f32: complex64 copy of the sources (S x N_z x n_t, made by the caller with launch_to_c64);
// MODE 1: xtr32 scratch for the trace forcing and vol32 for the volume (S x N_z x n_t)
cudaError_t launch_layer_solve_chunked(int mode, const Geometry& g, const LayerInfo* layers, int nloc_max, int K,
                                       const cf* Tm, const cf* Shi, const cf* Whi, const cf* Ehi, const cf* f32,
                                       const cd* xtr, cf* xtr32, cd* Y, size_t ystride, cd* out, cf* vol32,
                                       const int* flag, cf* bnd, int nsrc, int* status, cudaStream_t s) {
  if (nloc_max < 1 || nloc_max > kMaxNloc || nloc_max * kChunkQ > kChunkThreads || K < 1 || K > 64)
    return cudaErrorInvalidValue;
  cf* Yc = reinterpret_cast<cf*>(Y);
  const size_t smem = chunk_solve_smem(nloc_max);
  const dim3 grid(g.L * K, nsrc);
  const size_t T4n = (size_t)4 * (g.L - 1) * g.nt;
  cudaError_t e = cudaSuccess;
  if (mode == 1) {
    e = launch_to_c64(xtr, (size_t)nsrc * T4n, xtr32, s);
    if (e != cudaSuccess) return e;
  }
  auto go = [&](auto kern) {
    cudaError_t err = smem_limit_max(reinterpret_cast<const void*>(kern));
    if (err != cudaSuccess) return err;
    kern<<<grid, kChunkThreads, smem, s>>>(g, layers, K, Shi, Whi, Ehi, f32, xtr32, Yc, ystride, out, vol32, flag,
                                           nloc_max, bnd, status);
    return cudaGetLastError();
  };
  if (K > 1) {  // with one chunk the boundary values are zero and phase 1 has nothing to give
    e = mode == 0 ? go(layer_solve_chunk_kernel<0, 1>) : go(layer_solve_chunk_kernel<1, 1>);
    if (e != cudaSuccess) return e;
  }
  const size_t psmem = ((size_t)3 * K + 1) * nloc_max * sizeof(cf);
  e = smem_limit_max(reinterpret_cast<const void*>(chunk_propagate_kernel));
  if (e != cudaSuccess) return e;
  chunk_propagate_kernel<<<dim3(g.L, nsrc), kPropThreads, psmem, s>>>(g, layers, K, nloc_max, Tm, flag, mode, bnd);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = mode == 0 ? go(layer_solve_chunk_kernel<0, 3>) : go(layer_solve_chunk_kernel<1, 3>);
  if (e != cudaSuccess || mode == 0) return e;
  const size_t nv = (size_t)nsrc * g.Nz * g.nt;
  to_c128_kernel<<<(int)std::min<size_t>((nv + 255) / 256, 4096), 256, 0, s>>>(vol32, nv, out);
  return cudaGetLastError();
}

}  // namespace pt
