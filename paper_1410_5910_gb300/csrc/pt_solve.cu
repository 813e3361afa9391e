// Local solves (H^l)^{-1} (Algorithm 2, "solve local problems" and the
// reconstruction of Section 2.3) with the block factorization of the offline
// phase: forward  y_i = Sinv_i (f_i - W_i o y_{i-1}),
//         backward x_i = y_i - Sinv_i (E_i o x_{i+1}),   i = 0 .. n_t - 1,
// a chain of 2 n_t - 1 dependent nloc x nloc products.
//
// One thread-block cluster of kSolveCS CTAs per (layer, source): each CTA
// owns a slice of the nloc rows, computes its part of each product and
// stores it into every CTA's shared memory (distributed shared memory); one
// cluster barrier per step.  All global loads of step i+1 (Sinv entries,
// couplings, source / forcing values, stored forward iterates) are issued
// during step i, so the serial path holds only shared-memory traffic, the
// arithmetic and the barrier.
//
// Arithmetic: FP64 (layer_solve_kernel), or double-float
// (layer_solve_df_kernel below: Sinv stored as FP32 hi + lo, products and
// sums in FP32 pairs with error-free transformations, ~2^-45 relative), which
// moves the products off GB300's FP64 pipe.
#include <cooperative_groups.h>

#include "pt_common.cuh"

namespace cg = cooperative_groups;

namespace pt {

constexpr int kSolveCS = 8;                                              // CTAs per cluster
constexpr int kSolveRowsPerCta = (kMaxNloc + kSolveCS - 1) / kSolveCS;  // 15
constexpr int kSolveRW = (kSolveRowsPerCta + 7) / 8;                     // rows per warp: 2
constexpr int kSolveCW = (kMaxNloc + 31) / 32;                           // columns per lane: 4

__device__ __forceinline__ void ts(float a, float b, float& s, float& e) {
  s = a + b;
  float v = s - a;
  e = (a - (s - v)) + (b - v);
}
__device__ __forceinline__ void dfmac(float ah, float al, float xh, float xl, float& S, float& C) {
  float p = ah * xh;
  float pe = fmaf(ah, xh, -p);
  float s, e;
  ts(S, p, s, e);
  S = s;
  C += e + pe;
  C = fmaf(ah, xl, C);
  C = fmaf(al, xh, C);
}
__device__ __forceinline__ void df_shfl(float& S, float& C, int off) {
  float S2 = __shfl_down_sync(0xffffffffu, S, off);
  float C2 = __shfl_down_sync(0xffffffffu, C, off);
  float s, e;
  ts(S, S2, s, e);
  S = s;
  C = C + C2 + e;
}

// MODE 0: right-hand side, out = P b (trace vector), b = (-f, -f_0):
//   down rows of interface l: -N^l_n f, -N^l_{n+1} f; up rows of interface l-1: -N^l_0 f, -N^l_1 f.
// MODE 1: reconstruction, out = volume field; forcing f^l + (1/h^2)(row 1: +u_0,
//   row 0: -u_1, row n+1: -u_n, row n: +u_{n+1}) with u = u_down + u_up read from xtr.
template <int MODE, bool DF>
__global__ void __cluster_dims__(kSolveCS, 1, 1) __launch_bounds__(256)
    layer_solve_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cd* __restrict__ Sinv,
                       const cf* __restrict__ Shi, const cf* __restrict__ Slo, const cd* __restrict__ W,
                       const cd* __restrict__ E, const cd* __restrict__ f, const cd* __restrict__ xtr,
                       cd* __restrict__ Ystore, size_t ystride, cd* __restrict__ out, const int* __restrict__ nzflag) {
  __shared__ __align__(16) cd ybuf[2][kMaxNloc];
  __shared__ __align__(16) float4 vloc[kMaxNloc];  // FP64 mode: (re, im) as a double2 in the same 16 bytes
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
    return;  // uniform over the cluster, before any cluster barrier
  }

  const cd* fs = f + (size_t)s * g.Nz * nt;
  const cd* xs = (MODE == 1) ? xtr + (size_t)s * T4n : nullptr;
  cd* Y = Ystore + ((size_t)s * g.L + l) * ystride;
  const double ih2 = 1.0 / (g.h * g.h);
  const int nsteps = 2 * nt - 1;
  auto step_col = [&](int st) { return st < nt ? st : (nt - 2 - (st - nt)); };

  // ---- the role of this thread in the right-hand-side update: row rv = threadIdx.x
  const int rv = threadIdx.x;
  const bool vrow = rv < n;
  const bool in_layer = vrow && rv >= L.pad_top && rv < L.pad_top + L.n;
  const size_t frow = in_layer ? (size_t)(L.start + rv - L.pad_top) * nt : 0;
  // forcing of the reconstruction on the four trace rows: trace index and sign
  int ftr = -1;
  double fsg = 0.0;
  if (MODE == 1 && vrow) {
    if (L.has_top && rv == L.row[1]) { ftr = 2 * (l - 1); fsg = ih2; }
    if (L.has_top && rv == L.row[0]) { ftr = 2 * (l - 1) + 1; fsg = -ih2; }
    if (L.has_bot && rv == L.row[3]) { ftr = 2 * l; fsg = -ih2; }
    if (L.has_bot && rv == L.row[2]) { ftr = 2 * l + 1; fsg = ih2; }
  }

  // Prefetched operands of the next step.  Every load below is predicated
  // and its result is not selected against anything, so the thread does not
  // wait for it until the next step reads the register; predicates that are
  // false for a thread at every step leave the register at zero.
  cd p_sinv[kSolveRW][kSolveCW];
  cf p_hi[kSolveRW][kSolveCW], p_lo[kSolveRW][kSolveCW];
#pragma unroll
  for (int a = 0; a < kSolveRW; ++a)
#pragma unroll
    for (int c = 0; c < kSolveCW; ++c) {
      p_sinv[a][c] = make_double2(0, 0);
      p_hi[a][c] = make_float2(0.f, 0.f);
      p_lo[a][c] = make_float2(0.f, 0.f);
    }
  cd p_coef = make_double2(0, 0), p_f = make_double2(0, 0), p_ta = make_double2(0, 0), p_tb = make_double2(0, 0);
  cd p_y[kSolveRW];
#pragma unroll
  for (int a = 0; a < kSolveRW; ++a) p_y[a] = make_double2(0, 0);

  auto fetch = [&](int st) {
    const int i = step_col(st);
    const bool fwd = st < nt;
    const size_t base = L.sinv_off + (size_t)i * n * n;
#pragma unroll
    for (int a = 0; a < kSolveRW; ++a) {
      const int r = r0 + warp + 8 * a;
#pragma unroll
      for (int c = 0; c < kSolveCW; ++c) {
        const int k = lane + 32 * c;
        if (r < r1 && k < n) {
          if (DF) {
            p_hi[a][c] = __ldg(Shi + base + (size_t)r * n + k);
            p_lo[a][c] = __ldg(Slo + base + (size_t)r * n + k);
          } else {
            p_sinv[a][c] = __ldg(Sinv + base + (size_t)r * n + k);
          }
        }
      }
      if (!fwd && lane == 0 && r < r1) p_y[a] = Y[(size_t)i * n + r];
    }
    if (vrow) {
      const cd* cp = (fwd ? W : E) + L.coef_off + (size_t)i * n + rv;
      p_coef = __ldg(cp);
      if (fwd && in_layer) p_f = fs[frow + i];
      if (MODE == 1 && fwd && ftr >= 0) {
        p_ta = xs[(size_t)ftr * nt + i];
        p_tb = xs[(size_t)(T + ftr) * nt + i];
      }
    }
  };

  fetch(0);
  cluster.sync();  // every CTA of the cluster is resident before remote stores

  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < nt;
    const int i = step_col(st);
    // operands of this step (registers)
    cd c_sinv[kSolveRW][kSolveCW];
    cf c_hi[kSolveRW][kSolveCW], c_lo[kSolveRW][kSolveCW];
    cd c_y[kSolveRW];
#pragma unroll
    for (int a = 0; a < kSolveRW; ++a) {
#pragma unroll
      for (int c = 0; c < kSolveCW; ++c) {
        if (DF) { c_hi[a][c] = p_hi[a][c]; c_lo[a][c] = p_lo[a][c]; }
        else c_sinv[a][c] = p_sinv[a][c];
      }
      c_y[a] = p_y[a];
    }
    // v = f_i - W_i o y_{i-1} (forward)  |  v = E_i o x_{i+1} (backward); prev in the other buffer
    if (vrow) {
      const cd prev = ybuf[(i + 1) & 1][rv];
      cd v;
      if (fwd) {
        v = p_f;
        if (MODE == 1 && ftr >= 0) v = cadd(v, cscale(cadd(p_ta, p_tb), fsg));
        if (i > 0) v = csub(v, cmul(p_coef, prev));
      } else {
        v = cmul(p_coef, prev);
      }
      if (DF) {
        float rh = (float)v.x, ih = (float)v.y;
        vloc[rv] = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
      } else {
        reinterpret_cast<cd*>(vloc)[rv] = v;
      }
    }
    __syncthreads();
    if (st + 1 < nsteps) fetch(st + 1);
    cd* ycur = ybuf[i & 1];
#pragma unroll
    for (int a = 0; a < kSolveRW; ++a) {
      const int r = r0 + warp + 8 * a;
      cd acc;
      if (DF) {
        float Sr = 0.f, Cr = 0.f, Si = 0.f, Ci = 0.f;
#pragma unroll
        for (int c = 0; c < kSolveCW; ++c) {
          const int k = lane + 32 * c;
          if (k < n) {
            const float4 xv = vloc[k];
            const cf h = c_hi[a][c], lo = c_lo[a][c];
            dfmac(h.x, lo.x, xv.x, xv.z, Sr, Cr);
            dfmac(-h.y, -lo.y, xv.y, xv.w, Sr, Cr);
            dfmac(h.x, lo.x, xv.y, xv.w, Si, Ci);
            dfmac(h.y, lo.y, xv.x, xv.z, Si, Ci);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          df_shfl(Sr, Cr, o);
          df_shfl(Si, Ci, o);
        }
        acc = make_double2((double)Sr + (double)Cr, (double)Si + (double)Ci);
      } else {
        acc = make_double2(0, 0);
        const cd* vl = reinterpret_cast<const cd*>(vloc);
#pragma unroll
        for (int c = 0; c < kSolveCW; ++c) {
          const int k = lane + 32 * c;
          if (k < n) acc = cfma(c_sinv[a][c], vl[k], acc);
        }
        acc = warp_sum_cd(acc);
      }
      if (r < r1 && lane == 0) {
        const cd val = fwd ? acc : csub(c_y[a], acc);
        if (fwd) Y[(size_t)i * n + r] = val;
#pragma unroll
        for (int q = 0; q < kSolveCS; ++q) cluster.map_shared_rank(ycur, q)[r] = val;
        if (!fwd || i == nt - 1) {
          if (MODE == 0) {
            cd* b = out + (size_t)s * T4n;
            const cd mx = make_double2(-val.x, -val.y);
            if (L.has_bot && r == L.row[2]) b[(size_t)(2 * l) * nt + i] = mx;
            if (L.has_bot && r == L.row[3]) b[(size_t)(2 * l + 1) * nt + i] = mx;
            if (L.has_top && r == L.row[0]) b[(size_t)(T + 2 * (l - 1)) * nt + i] = mx;
            if (L.has_top && r == L.row[1]) b[(size_t)(T + 2 * (l - 1) + 1) * nt + i] = mx;
          } else if (r >= L.pad_top && r < L.pad_top + L.n) {
            out[(size_t)s * g.Nz * nt + (size_t)(L.start + r - L.pad_top) * nt + i] = val;
          }
        }
      }
    }
    cluster.sync();
  }
}

// ---------------------------------------------------------------------------
// Double-float local solve: the whole step runs in FP32 pairs (hi, lo).  The
// chain state, the couplings W/E and the stored forward iterates are kept as
// (re_hi, im_hi, re_lo, im_lo); only non-zero source and forcing values are
// converted from FP64 (a bit test, not an FP64 compare, decides) and only the
// emitted outputs are converted back, by one lane.  GB300 executes FP64
// arithmetic and FP64 conversions on its narrow FP64 pipe, so keeping them out
// of the per-step path is what makes the chain fast.
// ---------------------------------------------------------------------------
constexpr int kDfThreads = 512;  // 16 warps
constexpr int kDfCS = 4;         // CTAs per cluster (4 SMs per layer solve)
constexpr int kDfCW = (kMaxNloc + 31) / 32;

struct df2 {  // complex double-float, unevaluated sums re = rh + rl, im = ih + il
  float rh, ih, rl, il;
};
__device__ __forceinline__ float4 to4(df2 a) { return make_float4(a.rh, a.ih, a.rl, a.il); }
__device__ __forceinline__ df2 from4(float4 v) { return df2{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ bool nonzero_d(cd v) {
  return ((__double_as_longlong(v.x) | __double_as_longlong(v.y)) << 1) != 0;  // +-0 are zero
}
__device__ __forceinline__ df2 split_d(cd v) {
  float rh = (float)v.x, ih = (float)v.y;
  return df2{rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih)};
}
// normalise (S, C) into hi + lo with |lo| <= ulp(hi)/2
__device__ __forceinline__ void df_norm(float S, float C, float& hi, float& lo) {
  hi = S + C;
  lo = C - (hi - S);
}
// (Sr, Cr, Si, Ci) += a * x  (complex double-float multiply-accumulate)
__device__ __forceinline__ void df_cmac(float ahr, float ahi, float alr, float ali, df2 x, float& Sr, float& Cr,
                                        float& Si, float& Ci) {
  dfmac(ahr, alr, x.rh, x.rl, Sr, Cr);
  dfmac(-ahi, -ali, x.ih, x.il, Sr, Cr);
  dfmac(ahr, alr, x.ih, x.il, Si, Ci);
  dfmac(ahi, ali, x.rh, x.rl, Si, Ci);
}

// CS CTAs per cluster; a warp owns rows r0 + warp + 16 a, a < RW (independent chains interleave).
template <int MODE, int CS>
__global__ void __launch_bounds__(kDfThreads, 1)
    layer_solve_df_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cf* __restrict__ Shi,
                          const cf* __restrict__ Slo, const cf* __restrict__ Whi, const cf* __restrict__ Wlo,
                          const cf* __restrict__ Ehi, const cf* __restrict__ Elo, const cd* __restrict__ f,
                          const cd* __restrict__ xtr, float4* __restrict__ Ystore, size_t ystride,
                          cd* __restrict__ out, const int* __restrict__ nzflag) {
  __shared__ __align__(16) float4 ybuf[2][kMaxNloc];
  __shared__ __align__(16) float4 vloc[kMaxNloc];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int l = blockIdx.x / CS;
  const int s = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt;
  const int T = 2 * (g.L - 1);
  const size_t T4n = (size_t)2 * T * nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpc = (n + CS - 1) / CS;
  const int r0 = rank * rpc, r1 = min(n, r0 + rpc);
  constexpr int RW = ((kMaxNloc + CS - 1) / CS + 15) / 16;  // rows per warp

  if (MODE == 0 && nzflag[s * g.L + l] == 0) {
    cd* b = out + (size_t)s * T4n;
    for (int k = rank * blockDim.x + threadIdx.x; k < nt; k += CS * blockDim.x) {
      if (L.has_bot) {
        b[(size_t)(2 * l) * nt + k] = make_double2(0, 0);
        b[(size_t)(2 * l + 1) * nt + k] = make_double2(0, 0);
      }
      if (L.has_top) {
        b[(size_t)(T + 2 * (l - 1)) * nt + k] = make_double2(0, 0);
        b[(size_t)(T + 2 * (l - 1) + 1) * nt + k] = make_double2(0, 0);
      }
    }
    return;  // uniform over the cluster, before any cluster barrier
  }

  const cd* fs = f + (size_t)s * g.Nz * nt;
  const cd* xs = (MODE == 1) ? xtr + (size_t)s * T4n : nullptr;
  float4* Y = Ystore + ((size_t)s * g.L + l) * ystride;
  const double ih2 = 1.0 / (g.h * g.h);
  const int nsteps = 2 * nt - 1;
  auto step_col = [&](int st) { return st < nt ? st : (nt - 2 - (st - nt)); };

  const int rv = threadIdx.x;
  const bool vrow = rv < n;
  const bool in_layer = vrow && rv >= L.pad_top && rv < L.pad_top + L.n;
  const size_t frow = in_layer ? (size_t)(L.start + rv - L.pad_top) * nt : 0;
  int ftr = -1;
  double fsg = 0.0;
  if (MODE == 1 && vrow) {
    if (L.has_top && rv == L.row[1]) { ftr = 2 * (l - 1); fsg = ih2; }
    if (L.has_top && rv == L.row[0]) { ftr = 2 * (l - 1) + 1; fsg = -ih2; }
    if (L.has_bot && rv == L.row[3]) { ftr = 2 * l; fsg = -ih2; }
    if (L.has_bot && rv == L.row[2]) { ftr = 2 * l + 1; fsg = ih2; }
  }

  // prefetched operands of the next step (predicated loads, no selects on results)
  cf p_hi[RW][kDfCW], p_lo[RW][kDfCW];
  float4 p_y[RW];
#pragma unroll
  for (int a = 0; a < RW; ++a) {
    p_y[a] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < kDfCW; ++c) { p_hi[a][c] = make_float2(0.f, 0.f); p_lo[a][c] = make_float2(0.f, 0.f); }
  }
  cf p_ch = make_float2(0.f, 0.f), p_cl = make_float2(0.f, 0.f);
  cd p_f = make_double2(0, 0), p_ta = make_double2(0, 0), p_tb = make_double2(0, 0);
  auto fetch = [&](int st) {
    const int i = step_col(st);
    const bool fwd = st < nt;
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      const int r = r0 + warp + 16 * a;
      const bool rowok = r < r1;
      const size_t base = L.sinv_off + (size_t)i * n * n + (size_t)r * n;
#pragma unroll
      for (int c = 0; c < kDfCW; ++c) {
        const int k = lane + 32 * c;
        if (rowok && k < n) {
          p_hi[a][c] = __ldg(Shi + base + k);
          p_lo[a][c] = __ldg(Slo + base + k);
        }
      }
      if (!fwd && lane == 0 && rowok) p_y[a] = Y[(size_t)i * n + r];
    }
    if (vrow) {
      const size_t co = L.coef_off + (size_t)i * n + rv;
      p_ch = __ldg((fwd ? Whi : Ehi) + co);
      p_cl = __ldg((fwd ? Wlo : Elo) + co);
      if (fwd && in_layer) p_f = fs[frow + i];
      if (MODE == 1 && fwd && ftr >= 0) {
        p_ta = xs[(size_t)ftr * nt + i];
        p_tb = xs[(size_t)(T + ftr) * nt + i];
      }
    }
  };

  fetch(0);
  cluster.sync();

  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < nt;
    const int i = step_col(st);
    cf c_hi[RW][kDfCW], c_lo[RW][kDfCW];
    float4 c_y[RW];
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      c_y[a] = p_y[a];
#pragma unroll
      for (int c = 0; c < kDfCW; ++c) { c_hi[a][c] = p_hi[a][c]; c_lo[a][c] = p_lo[a][c]; }
    }
    // v = f_i - W_i o y_{i-1} (forward) | v = E_i o x_{i+1} (backward), in double-float
    if (vrow) {
      const df2 prev = from4(ybuf[(i + 1) & 1][rv]);
      float Sr = 0.f, Cr = 0.f, Si = 0.f, Ci = 0.f;
      if (fwd) {
        if (nonzero_d(p_f)) {
          const df2 fv = split_d(p_f);
          Sr = fv.rh; Cr = fv.rl; Si = fv.ih; Ci = fv.il;
        }
        if (MODE == 1 && ftr >= 0) {
          const df2 fv = split_d(cscale(cadd(p_ta, p_tb), fsg));
          float s1, e1;
          ts(Sr, fv.rh, s1, e1); Sr = s1; Cr += e1 + fv.rl;
          ts(Si, fv.ih, s1, e1); Si = s1; Ci += e1 + fv.il;
        }
        if (i > 0) df_cmac(-p_ch.x, -p_ch.y, -p_cl.x, -p_cl.y, prev, Sr, Cr, Si, Ci);
      } else {
        df_cmac(p_ch.x, p_ch.y, p_cl.x, p_cl.y, prev, Sr, Cr, Si, Ci);
      }
      df2 v;
      df_norm(Sr, Cr, v.rh, v.rl);
      df_norm(Si, Ci, v.ih, v.il);
      vloc[rv] = to4(v);
    }
    __syncthreads();
    if (st + 1 < nsteps) fetch(st + 1);
    float Sr[RW], Cr[RW], Si[RW], Ci[RW];
#pragma unroll
    for (int a = 0; a < RW; ++a) { Sr[a] = 0.f; Cr[a] = 0.f; Si[a] = 0.f; Ci[a] = 0.f; }
#pragma unroll
    for (int c = 0; c < kDfCW; ++c) {
      const int k = lane + 32 * c;
      if (k < n) {
        const df2 xv = from4(vloc[k]);
#pragma unroll
        for (int a = 0; a < RW; ++a)
          df_cmac(c_hi[a][c].x, c_hi[a][c].y, c_lo[a][c].x, c_lo[a][c].y, xv, Sr[a], Cr[a], Si[a], Ci[a]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int a = 0; a < RW; ++a) {
        df_shfl(Sr[a], Cr[a], o);
        df_shfl(Si[a], Ci[a], o);
      }
    }
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      const int r = r0 + warp + 16 * a;
      if (r < r1 && lane == 0) {
        df2 val;
        if (fwd) {
          df_norm(Sr[a], Cr[a], val.rh, val.rl);
          df_norm(Si[a], Ci[a], val.ih, val.il);
          Y[(size_t)i * n + r] = to4(val);
        } else {
          // x_i = y_i - acc
          float s1, e1;
          ts(c_y[a].x, -Sr[a], s1, e1);
          df_norm(s1, e1 + c_y[a].z - Cr[a], val.rh, val.rl);
          ts(c_y[a].y, -Si[a], s1, e1);
          df_norm(s1, e1 + c_y[a].w - Ci[a], val.ih, val.il);
        }
        float4* ycur = ybuf[i & 1];
        const float4 v4 = to4(val);
#pragma unroll
        for (int q = 0; q < CS; ++q) cluster.map_shared_rank(ycur, q)[r] = v4;
        if (!fwd || i == nt - 1) {
          if (MODE == 0) {
            const bool emit = (L.has_bot && (r == L.row[2] || r == L.row[3])) ||
                              (L.has_top && (r == L.row[0] || r == L.row[1]));
            if (emit) {
              cd* b = out + (size_t)s * T4n;
              const cd mx = make_double2(-((double)val.rh + (double)val.rl), -((double)val.ih + (double)val.il));
              if (L.has_bot && r == L.row[2]) b[(size_t)(2 * l) * nt + i] = mx;
              if (L.has_bot && r == L.row[3]) b[(size_t)(2 * l + 1) * nt + i] = mx;
              if (L.has_top && r == L.row[0]) b[(size_t)(T + 2 * (l - 1)) * nt + i] = mx;
              if (L.has_top && r == L.row[1]) b[(size_t)(T + 2 * (l - 1) + 1) * nt + i] = mx;
            }
          } else if (r >= L.pad_top && r < L.pad_top + L.n) {
            out[(size_t)s * g.Nz * nt + (size_t)(L.start + r - L.pad_top) * nt + i] =
                make_double2((double)val.rh + (double)val.rl, (double)val.ih + (double)val.il);
          }
        }
      }
    }
    cluster.sync();
  }
}

// ---------------------------------------------------------------------------
// FP32 single-source local solve, one CTA per (layer, source), no cluster.
// Sinv_i rounded to complex64 (the hi part of the double-float split) is
// copied into shared memory by one bulk asynchronous copy per column (the
// tensor-memory-access engine, completion on an mbarrier), double-buffered,
// while the previous column computes; four threads share a row (each a quarter
// of the columns, reduced with two shuffles) and the thread of quarter 0 keeps
// the row's chain state, so a step needs only CTA barriers.  Accuracy: FP32
// rounding carried through 2 n_t steps (about 1e-6 relative on the field).
// ---------------------------------------------------------------------------
constexpr int kF32Threads = 512;
constexpr int kF32Q = 4;  // threads per row

__device__ __forceinline__ uint32_t f32_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long f32_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for phase `parity` of an mbarrier, at most 2 s; false (and kErrTimeout) on expiry
__device__ __forceinline__ bool f32_mb_wait(uint64_t* bar, int parity, int* status) {
  const unsigned long long t0 = f32_timer();
  for (long long it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(f32_saddr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && f32_timer() - t0 > 2000000000ull) break;
  }
  atomicOr(status, kErrTimeout);
  return false;
}

// each Sinv buffer holds nloc_max^2 + 2 complex64 (one element of slack in front for a
// source block that starts 8 bytes off a 16-byte boundary, one at the end), rounded to an
// even count so that both buffers start on 16-byte boundaries (bulk-copy destinations)
__host__ __device__ inline size_t f32_buf_elems(int nloc_max) { return ((size_t)nloc_max * nloc_max + 3) & ~(size_t)1; }
size_t f32_solve_smem(int nloc_max) { return (2 * f32_buf_elems(nloc_max) + (size_t)kMaxNloc) * sizeof(cf); }

template <int MODE>
__global__ void __launch_bounds__(kF32Threads, 1)
    layer_solve_f32_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cf* __restrict__ Shi,
                           const cf* __restrict__ Whi, const cf* __restrict__ Ehi, const cd* __restrict__ f,
                           const cd* __restrict__ xtr, cf* __restrict__ Ystore, size_t ystride, cd* __restrict__ out,
                           const int* __restrict__ nzflag, int nmax, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  const int l = blockIdx.x, s = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt;
  const int T = 2 * (g.L - 1);
  const size_t T4n = (size_t)2 * T * nt;
  const size_t bufel = f32_buf_elems(nmax);  // even: B1 stays 16-byte aligned
  cf* B0 = reinterpret_cast<cf*>(smem);
  cf* B1 = B0 + bufel;
  cf* vloc = B1 + bufel;  // [kMaxNloc]
  const bool fnz = nzflag[s * g.L + l] != 0;

  if (MODE == 0 && !fnz) {
    cd* b = out + (size_t)s * T4n;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      if (L.has_bot) {
        b[(size_t)(2 * l) * nt + k] = make_double2(0, 0);
        b[(size_t)(2 * l + 1) * nt + k] = make_double2(0, 0);
      }
      if (L.has_top) {
        b[(size_t)(T + 2 * (l - 1)) * nt + k] = make_double2(0, 0);
        b[(size_t)(T + 2 * (l - 1) + 1) * nt + k] = make_double2(0, 0);
      }
    }
    return;
  }

  const int r = threadIdx.x / kF32Q, q = threadIdx.x % kF32Q;
  const bool own = r < n && q == 0;  // owner of row r's chain state
  const int chunk = (n + kF32Q - 1) / kF32Q;
  const int k0 = q * chunk, k1 = min(n, k0 + chunk);
  const cd* fs = f + (size_t)s * g.Nz * nt;
  const cd* xs = (MODE == 1) ? xtr + (size_t)s * T4n : nullptr;
  cf* Y = Ystore + ((size_t)s * g.L + l) * ystride;
  const int nsteps = 2 * nt - 1;
  auto col = [&](int st) { return st < nt ? st : nt - 2 - (st - nt); };
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
  // the source block of column i and where its element 0 sits in the buffer
  auto src_of = [&](int st) { return Shi + L.sinv_off + (size_t)col(st) * nn; };
  auto view_of = [&](int st) {
    cf* B = (st & 1) ? B1 : B0;
    return ((reinterpret_cast<uintptr_t>(src_of(st)) & 15) != 0) ? B + 1 : B;
  };

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(f32_saddr(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(f32_saddr(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // one thread: 16-byte aligned bulk part by the copy engine, an odd head / tail element by hand
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
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(f32_saddr(bb)), "r"(bytes)
                 : "memory");
    if (nbulk > 0)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              f32_saddr(view + head)),
          "l"(src + head), "r"(bytes), "r"(f32_saddr(bb))
          : "memory");
  };
  // per-row operands of a step, prefetched one step ahead by the row owner
  cf c_next = make_float2(0.f, 0.f), y_next = make_float2(0.f, 0.f);
  cd f_next = make_double2(0, 0), ta_next = make_double2(0, 0), tb_next = make_double2(0, 0);
  auto prefetch = [&](int st) {
    if (!own) return;
    const int i = col(st);
    const bool fwd = st < nt;
    c_next = __ldg((fwd ? Whi : Ehi) + L.coef_off + (size_t)i * n + r);
    if (fwd) {
      cd v = make_double2(0, 0);
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

  cf chain = make_float2(0.f, 0.f);  // y_{i-1} (forward) / x_{i+1} (backward) of row r
  stage(0);
  prefetch(0);
  for (int st = 0; st < nsteps; ++st) {
    const bool fwd = st < nt;
    const int i = col(st);
    const cf c = c_next, yst = y_next;
    const cd fv = f_next, ta = ta_next, tb = tb_next;
    if (st + 1 < nsteps) prefetch(st + 1);
    // (a) right-hand side of row r
    if (own) {
      float vr, vi;
      if (fwd) {
        cd d = fv;
        if (MODE == 1 && ftr >= 0) d = cadd(d, cscale(cadd(ta, tb), (double)fsg));
        vr = (float)d.x;
        vi = (float)d.y;
        if (i > 0) {
          vr -= c.x * chain.x - c.y * chain.y;
          vi -= c.x * chain.y + c.y * chain.x;
        }
      } else {
        vr = c.x * chain.x - c.y * chain.y;
        vi = c.x * chain.y + c.y * chain.x;
      }
      vloc[r] = make_float2(vr, vi);
    }
    // Sinv_i in shared memory: phase (st / 2) of the buffer's barrier (bounded wait)
    if (!f32_mb_wait(&bar[st & 1], (st >> 1) & 1, status)) return;
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
      }
      if (!fwd || i == nt - 1) {
        if (MODE == 0) {
          if (emit >= 0) out[(size_t)s * T4n + (size_t)emit * nt + i] = make_double2(-(double)chain.x, -(double)chain.y);
        } else if (in_layer) {
          out[(size_t)s * g.Nz * nt + frow + i] = make_double2((double)chain.x, (double)chain.y);
        }
      }
    }
    __syncthreads();  // vloc is rewritten in the next step
  }
}

// ---------------------------------------------------------------------------
// FP32 local solve on a cluster of CS CTAs per (layer, source): CTA c owns the
// rows [c rpc, (c + 1) rpc) of the local problem, copies only its rows of each
// column's Schur inverse (one bulk copy per column and CTA, double-buffered)
// and computes only their products; the owners of the right-hand-side entries
// v_r broadcast them to every CTA of the cluster through distributed shared
// memory (double-buffered by step parity), one cluster barrier per step.
// The per-row operands of the next step are loaded after the barrier, so its
// release never waits for loads in flight.
// ---------------------------------------------------------------------------
constexpr int kF32cQ = 8;         // threads per row
constexpr int kF32cThreads = 256;

template <int CS>
struct F32cLayout {
  static constexpr int RPC = (kMaxNloc + CS - 1) / CS;
  // Sinv slice buffers: RPC * kMaxNloc + 2 complex64 each, even count (16-byte aligned)
  static constexpr size_t buf = ((size_t)RPC * kMaxNloc + 3) & ~(size_t)1;
  static constexpr size_t bytes = (2 * buf + 2 * (size_t)kMaxNloc) * sizeof(cf);
};

template <int MODE, int CS>
__global__ void __launch_bounds__(kF32cThreads, 1)
    layer_solve_f32c_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cf* __restrict__ Shi,
                            const cf* __restrict__ Whi, const cf* __restrict__ Ehi, const cd* __restrict__ f,
                            const cd* __restrict__ xtr, cf* __restrict__ Ystore, size_t ystride,
                            cd* __restrict__ out, const int* __restrict__ nzflag, const int* __restrict__ firstcol,
                            int* __restrict__ status) {
  using Lay = F32cLayout<CS>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int l = blockIdx.x / CS, s = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt;
  const int T = 2 * (g.L - 1);
  const size_t T4n = (size_t)2 * T * nt;
  cf* B0 = reinterpret_cast<cf*>(smem);
  cf* B1 = B0 + Lay::buf;
  cf* vbuf = B1 + Lay::buf;  // [2][kMaxNloc], written by every CTA of the cluster
  const bool fnz = nzflag[s * g.L + l] != 0;
  const int rpc = (n + CS - 1) / CS;
  const int r0 = rank * rpc, r1 = min(n, r0 + rpc);

  if (MODE == 0 && !fnz) {  // uniform over the cluster, before any cluster barrier
    cd* b = out + (size_t)s * T4n;
    for (int k = rank * blockDim.x + threadIdx.x; k < nt; k += CS * blockDim.x) {
      if (L.has_bot) {
        b[(size_t)(2 * l) * nt + k] = make_double2(0, 0);
        b[(size_t)(2 * l + 1) * nt + k] = make_double2(0, 0);
      }
      if (L.has_top) {
        b[(size_t)(T + 2 * (l - 1)) * nt + k] = make_double2(0, 0);
        b[(size_t)(T + 2 * (l - 1) + 1) * nt + k] = make_double2(0, 0);
      }
    }
    return;
  }

  const int lr = threadIdx.x / kF32cQ, q = threadIdx.x % kF32cQ;  // local row, column chunk
  const int r = r0 + lr;
  const bool own = r < r1 && q == 0;
  const int chunk = (n + kF32cQ - 1) / kF32cQ;
  const int k0 = q * chunk, k1 = min(n, k0 + chunk);
  const cd* fs = f + (size_t)s * g.Nz * nt;
  const cd* xs = (MODE == 1) ? xtr + (size_t)s * T4n : nullptr;
  cf* Y = Ystore + ((size_t)s * g.L + l) * ystride;
  const int nsteps = 2 * nt - 1;
  auto col = [&](int st) { return st < nt ? st : nt - 2 - (st - nt); };
  // right-hand side of point sources: the forward iterates vanish before the first column
  // with a non-zero source entry, so the chain starts there (stored iterates read as zero)
  const int st0 = (MODE == 0 && firstcol) ? min(firstcol[s * g.L + l], nt - 1) : 0;
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
  int emit = -1;
  if (MODE == 0 && own) {
    if (L.has_bot && r == L.row[2]) emit = 2 * l;
    if (L.has_bot && r == L.row[3]) emit = 2 * l + 1;
    if (L.has_top && r == L.row[0]) emit = T + 2 * (l - 1);
    if (L.has_top && r == L.row[1]) emit = T + 2 * (l - 1) + 1;
  }
  const int cnt = (r1 - r0) * n;  // this CTA's slice of a column: contiguous rows r0 .. r1 - 1
  auto src_of = [&](int st) { return Shi + L.sinv_off + (size_t)col(st) * n * n + (size_t)r0 * n; };
  auto view_of = [&](int st) {
    cf* B = ((st - st0) & 1) ? B1 : B0;
    return ((reinterpret_cast<uintptr_t>(src_of(st)) & 15) != 0) ? B + 1 : B;
  };
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(f32_saddr(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(f32_saddr(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // every call arms the buffer's barrier (zero bytes for a CTA that owns no rows)
  auto stage = [&](int st) {
    if (threadIdx.x != 0) return;
    const cf* src = src_of(st);
    cf* view = view_of(st);
    const int head = (cnt > 0 && (reinterpret_cast<uintptr_t>(src) & 15)) ? 1 : 0;
    const int m = cnt > 0 ? cnt - head : 0;
    const int nbulk = m & ~1;
    if (head) view[0] = src[0];
    if (m & 1) view[cnt - 1] = src[cnt - 1];
    uint64_t* bb = &bar[(st - st0) & 1];
    const uint32_t bytes = (uint32_t)nbulk * (uint32_t)sizeof(cf);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(f32_saddr(bb)), "r"(bytes)
                 : "memory");
    if (nbulk > 0)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              f32_saddr(view + head)),
          "l"(src + head), "r"(bytes), "r"(f32_saddr(bb))
          : "memory");
  };
  cf c_next = make_float2(0.f, 0.f), y_next = make_float2(0.f, 0.f);
  cd f_next = make_double2(0, 0), ta_next = make_double2(0, 0), tb_next = make_double2(0, 0);
  auto prefetch = [&](int st) {
    if (!own) return;
    const int i = col(st);
    const bool fwd = st < nt;
    c_next = __ldg((fwd ? Whi : Ehi) + L.coef_off + (size_t)i * n + r);
    if (fwd) {
      cd v = make_double2(0, 0);
      if (fnz && in_layer) v = fs[frow + i];
      f_next = v;
      if (MODE == 1 && ftr >= 0) {
        ta_next = xs[(size_t)ftr * nt + i];
        tb_next = xs[(size_t)(T + ftr) * nt + i];
      }
    } else {
      cf y = make_float2(0.f, 0.f);
      if (i >= st0) y = Y[(size_t)i * n + r];
      y_next = y;
    }
  };

  cf chain = make_float2(0.f, 0.f);
  // Global stores of a step (the stored forward iterate, the output) are issued after the
  // next step's cluster barrier, so that barrier's release does not wait for them
  int pend_i = -1;
  bool pend_fwd = false;
  auto flush = [&]() {
    if (!own || pend_i < 0) return;
    const int i = pend_i;
    if (pend_fwd) Y[(size_t)i * n + r] = chain;
    if (!pend_fwd || i == nt - 1) {
      if (MODE == 0) {
        if (emit >= 0) out[(size_t)s * T4n + (size_t)emit * nt + i] = make_double2(-(double)chain.x, -(double)chain.y);
      } else if (in_layer) {
        out[(size_t)s * g.Nz * nt + frow + i] = make_double2((double)chain.x, (double)chain.y);
      }
    }
    pend_i = -1;
  };
  // after a timed-out wait the CTA stops computing but keeps taking part in every
  // cluster barrier, so its peers are never left waiting; the error is in *status
  bool alive = true;
  __syncthreads();  // mbarriers initialised
  stage(st0);
  prefetch(st0);
  cluster.sync();  // every CTA of the cluster is resident before remote stores
  for (int st = st0; st < nsteps; ++st) {
    const bool fwd = st < nt;
    const int i = col(st);
    const int t = st - st0;  // local step: buffer and barrier-phase parity
    cf* vb = vbuf + (t & 1) * kMaxNloc;
    // (a) right-hand side of my rows, broadcast to every CTA of the cluster
    if (own) {
      const cf c = c_next;
      float vr, vi;
      if (fwd) {
        cd d = f_next;
        if (MODE == 1 && ftr >= 0) d = cadd(d, cscale(cadd(ta_next, tb_next), (double)fsg));
        vr = (float)d.x;
        vi = (float)d.y;
        if (i > 0) {
          vr -= c.x * chain.x - c.y * chain.y;
          vi -= c.x * chain.y + c.y * chain.x;
        }
      } else {
        vr = c.x * chain.x - c.y * chain.y;
        vi = c.x * chain.y + c.y * chain.x;
      }
      const cf v = make_float2(vr, vi);
#pragma unroll
      for (int p = 0; p < CS; ++p) cluster.map_shared_rank(vb, p)[r] = v;
    }
    const cf yst = y_next;
    cluster.sync();  // v complete in every CTA; this CTA's reads of step st - 1 are over
    flush();         // the previous step's global stores
    if (alive && st + 1 < nsteps) {
      stage(st + 1);     // the other buffer was last read in step st - 1
      prefetch(st + 1);  // consumed before the next barrier
    }
    if (alive) alive = __all_sync(0xffffffffu, f32_mb_wait(&bar[t & 1], (t >> 1) & 1, status));
    if (!alive) continue;
    // (b) my rows of Sinv_i v
    const cf* Srow = view_of(st) + (size_t)min(lr, max(r1 - r0 - 1, 0)) * n;
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      const cf a0 = Srow[k], a1 = Srow[k + 1];
      const cf v0 = vb[k], v1 = vb[k + 1];
      ar = fmaf(a0.x, v0.x, ar); ar = fmaf(-a0.y, v0.y, ar);
      ai = fmaf(a0.x, v0.y, ai); ai = fmaf(a0.y, v0.x, ai);
      br = fmaf(a1.x, v1.x, br); br = fmaf(-a1.y, v1.y, br);
      bi = fmaf(a1.x, v1.y, bi); bi = fmaf(a1.y, v1.x, bi);
    }
    if (k < k1) {
      const cf a0 = Srow[k], v0 = vb[k];
      ar = fmaf(a0.x, v0.x, ar); ar = fmaf(-a0.y, v0.y, ar);
      ai = fmaf(a0.x, v0.y, ai); ai = fmaf(a0.y, v0.x, ai);
    }
    ar += br;
    ai += bi;
#pragma unroll
    for (int o = 1; o < kF32cQ; o <<= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (own) {
      chain = fwd ? make_float2(ar, ai) : make_float2(yst.x - ar, yst.y - ai);
      pend_i = i;
      pend_fwd = fwd;
    }
  }
  flush();
  cluster.sync();  // no CTA leaves while a peer may still write its shared memory
}

// FP32 single-source local solves: cluster = 4 or 8 CTAs per (layer, source), else one CTA
cudaError_t launch_layer_solve_f32(int mode, const Geometry& g, const LayerInfo* layers, int nloc_max, const cf* Shi,
                                   const cf* Whi, const cf* Ehi, const cd* f, const cd* xtr, cd* Y, size_t ystride,
                                   cd* out, const int* flag, const int* firstcol, int nsrc, int* status, int cluster,
                                   cudaStream_t s) {
  if (nloc_max < 1 || nloc_max > kMaxNloc || nloc_max * kF32Q > kF32Threads) return cudaErrorInvalidValue;
  cf* Yc = reinterpret_cast<cf*>(Y);
  cudaError_t e;
  if (cluster == 4 || cluster == 8) {
    static_assert(F32cLayout<4>::RPC * kF32cQ <= kF32cThreads, "rows x threads per row");
    auto go = [&](auto kern, int CS, size_t smem) {
      cudaError_t err = smem_limit_max(reinterpret_cast<const void*>(kern));
      if (err != cudaSuccess) return err;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(CS * g.L, nsrc);
      cfg.blockDim = dim3(kF32cThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, kern, g, layers, Shi, Whi, Ehi, f, xtr, Yc, ystride, out, flag, firstcol,
                                status);
    };
    if (cluster == 4)
      e = mode == 0 ? go(layer_solve_f32c_kernel<0, 4>, 4, F32cLayout<4>::bytes)
                    : go(layer_solve_f32c_kernel<1, 4>, 4, F32cLayout<4>::bytes);
    else
      e = mode == 0 ? go(layer_solve_f32c_kernel<0, 8>, 8, F32cLayout<8>::bytes)
                    : go(layer_solve_f32c_kernel<1, 8>, 8, F32cLayout<8>::bytes);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  const size_t smem = f32_solve_smem(nloc_max);
  dim3 grid(g.L, nsrc);
  if (mode == 0) {
    e = smem_limit_max(reinterpret_cast<const void*>(layer_solve_f32_kernel<0>));
    if (e != cudaSuccess) return e;
    layer_solve_f32_kernel<0><<<grid, kF32Threads, smem, s>>>(g, layers, Shi, Whi, Ehi, f, xtr, Yc, ystride, out, flag,
                                                              nloc_max, status);
  } else {
    e = smem_limit_max(reinterpret_cast<const void*>(layer_solve_f32_kernel<1>));
    if (e != cudaSuccess) return e;
    layer_solve_f32_kernel<1><<<grid, kF32Threads, smem, s>>>(g, layers, Shi, Whi, Ehi, f, xtr, Yc, ystride, out, flag,
                                                              nloc_max, status);
  }
  return cudaGetLastError();
}

// flag[s * L + l] = 1 when f^l of source s has a non-zero entry; first (optional) = the
// first grid column with one (n_t when none): the forward substitution is zero before it.
// 1024 threads, eight loads in flight per thread (a layer of the 511 x 1023 workload is
// 36 K entries: about five round trips).
constexpr int kNzThreads = 1024;
constexpr int kNzUnroll = 8;

__global__ void __launch_bounds__(kNzThreads) layer_nonzero_kernel(Geometry g, const LayerInfo* __restrict__ layers,
                                                                   const cd* __restrict__ f, int* __restrict__ flag,
                                                                   int* __restrict__ first) {
  const LayerInfo L = layers[blockIdx.x];
  const int s = blockIdx.y;
  const cd* fs = f + (size_t)s * g.Nz * g.nt + (size_t)L.start * g.nt;
  const size_t total = (size_t)L.n * g.nt;
  int nz = 0, fc = g.nt;
  for (size_t base = 0; base < total; base += (size_t)kNzThreads * kNzUnroll) {
    cd v[kNzUnroll];
#pragma unroll
    for (int u = 0; u < kNzUnroll; ++u) {
      const size_t k = base + (size_t)u * kNzThreads + threadIdx.x;
      v[u] = k < total ? __ldg(fs + k) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < kNzUnroll; ++u) {
      const size_t k = base + (size_t)u * kNzThreads + threadIdx.x;
      if (v[u].x != 0.0 || v[u].y != 0.0) {
        nz = 1;
        fc = min(fc, (int)(k % g.nt));
      }
    }
  }
  nz = __syncthreads_or(nz);
  __shared__ int smin;
  if (threadIdx.x == 0) smin = g.nt;
  __syncthreads();
  if (fc < g.nt) atomicMin(&smin, fc);
  __syncthreads();
  if (threadIdx.x == 0) {
    flag[s * g.L + blockIdx.x] = nz;
    if (first) first[s * g.L + blockIdx.x] = smin;
  }
}

__global__ void split_sinv_kernel(const cd* __restrict__ src, size_t n, cf* __restrict__ hi, cf* __restrict__ lo) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    cd v = src[q];
    cf h = make_float2((float)v.x, (float)v.y);
    hi[q] = h;
    lo[q] = make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
  }
}

cudaError_t launch_layer_nonzero(const Geometry& g, const LayerInfo* layers, const cd* f, int* flag, int* first,
                                 int nsrc, cudaStream_t s) {
  layer_nonzero_kernel<<<dim3(g.L, nsrc), kNzThreads, 0, s>>>(g, layers, f, flag, first);
  return cudaGetLastError();
}

// df: use the double-float (hi, lo) factors instead of the FP64 ones
cudaError_t launch_layer_solve2(int mode, bool /*df*/, const Geometry& g, const LayerInfo* layers, const cd* Sinv,
                                const cf* Shi, const cf* Slo, const cd* W, const cd* E, const cd* f, const cd* xtr,
                                cd* Y, size_t ystride, cd* out, const int* flag, int nsrc, cudaStream_t s) {
  dim3 grid(kSolveCS * g.L, nsrc);
  if (mode == 0)
    layer_solve_kernel<0, false><<<grid, 256, 0, s>>>(g, layers, Sinv, Shi, Slo, W, E, f, xtr, Y, ystride, out, flag);
  else
    layer_solve_kernel<1, false><<<grid, 256, 0, s>>>(g, layers, Sinv, Shi, Slo, W, E, f, xtr, Y, ystride, out, flag);
  return cudaGetLastError();
}

// FP64 factors (the entry point used by the plain path and pt_rhs_noalloc)
cudaError_t launch_layer_solve(int mode, const Geometry& g, const LayerInfo* layers, const cd* Sinv, const cd* W,
                               const cd* E, const cd* f, const cd* xtr, cd* Y, size_t ystride, cd* out,
                               const int* flag, int nsrc, cudaStream_t s) {
  return launch_layer_solve2(mode, false, g, layers, Sinv, nullptr, nullptr, W, E, f, xtr, Y, ystride, out, flag,
                             nsrc, s);
}

cudaError_t launch_layer_solve_df(int mode, const Geometry& g, const LayerInfo* layers, const cf* Shi, const cf* Slo,
                                  const cf* Whi, const cf* Wlo, const cf* Ehi, const cf* Elo, const cd* f,
                                  const cd* xtr, cd* Y, size_t ystride, cd* out, const int* flag, int nsrc,
                                  cudaStream_t s) {
  static_assert(sizeof(float4) == sizeof(cd), "double-float iterates reuse the FP64 scratch layout");
  float4* Y4 = reinterpret_cast<float4*>(Y);
  auto go = [&](auto kern, int cs) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * g.L, nsrc);
    cfg.blockDim = dim3(kDfThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g, layers, Shi, Slo, Whi, Wlo, Ehi, Elo, f, xtr, Y4, ystride, out, flag);
  };
  cudaError_t e = mode == 0 ? go(layer_solve_df_kernel<0, kDfCS>, kDfCS) : go(layer_solve_df_kernel<1, kDfCS>, kDfCS);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_split_sinv(const cd* src, size_t n, cf* hi, cf* lo, cudaStream_t s) {
  split_sinv_kernel<<<1216, 256, 0, s>>>(src, n, hi, lo);
  return cudaGetLastError();
}

}  // namespace pt
