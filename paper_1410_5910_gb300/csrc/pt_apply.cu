// Block-sparse trace operators of the permuted polarized jump system.
//
// Each output trace of P M = D + R (Definition 9 and the splitting of
// Section 3.5), of R, or of one step of the sweeps D_down^{-1} / D_up^{-1}
// (Section 4.1) is a sum of at most four n_t x n_t block products, each
// applied to one input trace or to the sum of two, plus identity terms:
//
//   y[out] = alpha * ( sum_t sign_t B_t (x[in1_t] + x[in2_t]) + sum_e sign_e src_e[trace_e] )
//            + beta * aux[out].
//
// Three arithmetic modes:
//   FP64  blocks in complex128, FP64 multiply-add (bound by the FP64 pipe on GB300);
//   FP32  blocks in complex64, FP32 multiply-add (bound by HBM);
//   DF    blocks as two complex64 arrays hi + lo (hi = fl32(b), lo = fl32(b - hi)),
//         products and sums in double-float arithmetic: exact products of the
//         high parts (FMA), error-free two-sum accumulation, cross terms in a
//         compensation word.  About 2^-45 relative accuracy, FP32 pipes, HBM bound.
// A CTA computes rows_per_cta consecutive rows of one output trace for one
// source; inputs are staged in shared memory once per CTA.  The grid runs the
// sources fastest so that a batch of sources shares each block row through L2.
#include "pt_common.cuh"

namespace pt {

enum ApplyMode { kFP64 = 0, kFP32 = 1, kDF = 2 };

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float v = s - a;
  e = (a - (s - v)) + (b - v);
}
// (S, C) += (ah + al) * (xh + xl), dropping al * xl
__device__ __forceinline__ void df_mac(float ah, float al, float xh, float xl, float& S, float& C) {
  float p = ah * xh;
  float pe = fmaf(ah, xh, -p);  // exact error of the product
  float s, e;
  two_sum(S, p, s, e);
  S = s;
  C += e + pe;
  C = fmaf(ah, xl, C);
  C = fmaf(al, xh, C);
}
__device__ __forceinline__ void df_shfl_add(float& S, float& C, int off) {
  float S2 = __shfl_down_sync(0xffffffffu, S, off);
  float C2 = __shfl_down_sync(0xffffffffu, C, off);
  float s, e;
  two_sum(S, S2, s, e);
  S = s;
  C = C + C2 + e;
}

template <int MODE>
__global__ void __launch_bounds__(256) apply_kernel(int nt, int ld, int T4, const ApplyRow* __restrict__ table,
                                                    const void* __restrict__ blocks_a,
                                                    const void* __restrict__ blocks_b, const cd* x,
                                                    const cd* __restrict__ aux, cd* y, int rows_per_cta,
                                                    double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ApplyRow row;
  if (threadIdx.x == 0) row = table[blockIdx.z];
  __syncthreads();
  const int s = blockIdx.x;
  const size_t vs = (size_t)T4 * nt;
  const cd* xs = x + s * vs;
  const cd* as = aux ? aux + s * vs : nullptr;
  const size_t bsz = (size_t)nt * ld;
  const int nterms = row.nterms;

  // ---- stage sign_t (x[in1] + x[in2]) for every term, padded with zeros to ld
  for (int t = 0; t < nterms; ++t) {
    const ApplyTerm tm = row.t[t];
    const cd* a = xs + (size_t)tm.in1 * nt;
    const cd* b = tm.in2 >= 0 ? xs + (size_t)tm.in2 * nt : nullptr;
    for (int k = threadIdx.x; k < ld; k += blockDim.x) {
      cd v = make_double2(0, 0);
      if (k < nt) {
        v = a[k];
        if (b) v = cadd(v, b[k]);
        v = cscale(v, tm.sign);
      }
      if (MODE == kFP64) {
        reinterpret_cast<cd*>(smem_raw)[t * ld + k] = v;
      } else if (MODE == kFP32) {
        reinterpret_cast<cf*>(smem_raw)[t * ld + k] = make_float2((float)v.x, (float)v.y);
      } else {
        float rh = (float)v.x, ih = (float)v.y;
        float rl = (float)(v.x - (double)rh), il = (float)(v.y - (double)ih);
        reinterpret_cast<float4*>(smem_raw)[t * ld + k] = make_float4(rh, ih, rl, il);
      }
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.y * rows_per_cta;
  for (int rr = warp; rr < rows_per_cta; rr += 8) {
    const int r = r0 + rr;
    if (r >= nt) break;
    cd val;
    if (MODE == kFP64) {
      const cd* xin = reinterpret_cast<const cd*>(smem_raw);
      cd acc = make_double2(0, 0);
      for (int t = 0; t < nterms; ++t) {
        const cd* B = static_cast<const cd*>(blocks_a) + (size_t)row.t[t].block * bsz + (size_t)r * ld;
        const cd* xv = xin + t * ld;
        int k = lane;
        for (; k + 96 < nt; k += 128) {
          cd b0 = __ldg(B + k), b1 = __ldg(B + k + 32), b2 = __ldg(B + k + 64), b3 = __ldg(B + k + 96);
          acc = cfma(b0, xv[k], acc);
          acc = cfma(b1, xv[k + 32], acc);
          acc = cfma(b2, xv[k + 64], acc);
          acc = cfma(b3, xv[k + 96], acc);
        }
        for (; k < nt; k += 32) acc = cfma(__ldg(B + k), xv[k], acc);
      }
      val = warp_sum_cd(acc);
    } else if (MODE == kFP32) {
      const float4* xin = reinterpret_cast<const float4*>(smem_raw);  // two complex64 per float4
      float are = 0.f, aim = 0.f;
      const int np = ld >> 1;
      for (int t = 0; t < nterms; ++t) {
        const float4* B = reinterpret_cast<const float4*>(static_cast<const cf*>(blocks_a) +
                                                          (size_t)row.t[t].block * bsz + (size_t)r * ld);
        const float4* xv = xin + t * np;
        int k = lane;
        for (; k + 96 < np; k += 128) {
          float4 b[4], v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) b[u] = __ldg(B + k + 32 * u);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            v[u] = xv[k + 32 * u];
            are = fmaf(b[u].x, v[u].x, are);
            are = fmaf(-b[u].y, v[u].y, are);
            are = fmaf(b[u].z, v[u].z, are);
            are = fmaf(-b[u].w, v[u].w, are);
            aim = fmaf(b[u].x, v[u].y, aim);
            aim = fmaf(b[u].y, v[u].x, aim);
            aim = fmaf(b[u].z, v[u].w, aim);
            aim = fmaf(b[u].w, v[u].z, aim);
          }
        }
        for (; k < np; k += 32) {
          float4 b = __ldg(B + k), v = xv[k];
          are = fmaf(b.x, v.x, are);
          are = fmaf(-b.y, v.y, are);
          are = fmaf(b.z, v.z, are);
          are = fmaf(-b.w, v.w, are);
          aim = fmaf(b.x, v.y, aim);
          aim = fmaf(b.y, v.x, aim);
          aim = fmaf(b.z, v.w, aim);
          aim = fmaf(b.w, v.z, aim);
        }
      }
      cf acc = warp_sum_cf(make_float2(are, aim));
      val = make_double2(acc.x, acc.y);
    } else {
      const float4* xin = reinterpret_cast<const float4*>(smem_raw);  // (re_hi, im_hi, re_lo, im_lo)
      // two independent accumulator sets (even / odd column pairs of a lane) halve the
      // dependent two-sum chains; they are merged error-free at the end
      float Sr = 0.f, Cr = 0.f, Si = 0.f, Ci = 0.f;
      float Sr2 = 0.f, Cr2 = 0.f, Si2 = 0.f, Ci2 = 0.f;
      const int np = ld >> 1;
      for (int t = 0; t < nterms; ++t) {
        const size_t off = (size_t)row.t[t].block * bsz + (size_t)r * ld;
        const float4* H = reinterpret_cast<const float4*>(static_cast<const cf*>(blocks_a) + off);
        const float4* Lo = reinterpret_cast<const float4*>(static_cast<const cf*>(blocks_b) + off);
        const float4* xv = xin + t * ld;
        int k = lane;
        for (; k + 32 < np; k += 64) {
          const float4 h0 = __ldg(H + k), l0 = __ldg(Lo + k), h1 = __ldg(H + k + 32), l1 = __ldg(Lo + k + 32);
          const float4 a0 = xv[2 * k], a1 = xv[2 * k + 1];
          const float4 b0 = xv[2 * (k + 32)], b1 = xv[2 * (k + 32) + 1];
          df_mac(h0.x, l0.x, a0.x, a0.z, Sr, Cr);
          df_mac(h1.x, l1.x, b0.x, b0.z, Sr2, Cr2);
          df_mac(h0.x, l0.x, a0.y, a0.w, Si, Ci);
          df_mac(h1.x, l1.x, b0.y, b0.w, Si2, Ci2);
          df_mac(-h0.y, -l0.y, a0.y, a0.w, Sr, Cr);
          df_mac(-h1.y, -l1.y, b0.y, b0.w, Sr2, Cr2);
          df_mac(h0.y, l0.y, a0.x, a0.z, Si, Ci);
          df_mac(h1.y, l1.y, b0.x, b0.z, Si2, Ci2);
          df_mac(h0.z, l0.z, a1.x, a1.z, Sr, Cr);
          df_mac(h1.z, l1.z, b1.x, b1.z, Sr2, Cr2);
          df_mac(h0.z, l0.z, a1.y, a1.w, Si, Ci);
          df_mac(h1.z, l1.z, b1.y, b1.w, Si2, Ci2);
          df_mac(-h0.w, -l0.w, a1.y, a1.w, Sr, Cr);
          df_mac(-h1.w, -l1.w, b1.y, b1.w, Sr2, Cr2);
          df_mac(h0.w, l0.w, a1.x, a1.z, Si, Ci);
          df_mac(h1.w, l1.w, b1.x, b1.z, Si2, Ci2);
        }
        for (; k < np; k += 32) {
          const float4 h = __ldg(H + k), l = __ldg(Lo + k);
          const float4 x0 = xv[2 * k], x1 = xv[2 * k + 1];
          df_mac(h.x, l.x, x0.x, x0.z, Sr, Cr);
          df_mac(-h.y, -l.y, x0.y, x0.w, Sr, Cr);
          df_mac(h.x, l.x, x0.y, x0.w, Si, Ci);
          df_mac(h.y, l.y, x0.x, x0.z, Si, Ci);
          df_mac(h.z, l.z, x1.x, x1.z, Sr, Cr);
          df_mac(-h.w, -l.w, x1.y, x1.w, Sr, Cr);
          df_mac(h.z, l.z, x1.y, x1.w, Si, Ci);
          df_mac(h.w, l.w, x1.x, x1.z, Si, Ci);
        }
      }
      {  // merge the second set: (S, C) += (S2, C2)
        float s1, e1;
        two_sum(Sr, Sr2, s1, e1);
        Sr = s1;
        Cr = Cr + Cr2 + e1;
        two_sum(Si, Si2, s1, e1);
        Si = s1;
        Ci = Ci + Ci2 + e1;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        df_shfl_add(Sr, Cr, o);
        df_shfl_add(Si, Ci, o);
      }
      val = make_double2((double)Sr + (double)Cr, (double)Si + (double)Ci);
    }
    if (lane == 0) {
      for (int e = 0; e < row.nid; ++e) {
        const cd* src = row.id_src[e] == 0 ? xs : as;
        val = cadd(val, cscale(src[(size_t)row.id_trace[e] * nt + r], row.id_sign[e]));
      }
      val = cscale(val, alpha);
      if (beta != 0.0) val = cadd(val, cscale(as[(size_t)row.out * nt + r], beta));
      y[s * vs + (size_t)row.out * nt + r] = val;
    }
  }
}

// ---- FP32 sweep steps: one row per warp, whole block rows in flight ---------------
// A sweep step (Section 4.1) is small (8 blocks): the time is memory latency, not
// bandwidth.  Each lane issues the loads of its share of both terms' block rows into
// registers first (up to MAXC float4 = 2 complex64 each per term), then the CTA stages
// the input traces, so the two latencies overlap and a row costs one round trip.
template <int MAXC>
__global__ void __launch_bounds__(256) apply_f32_rows_kernel(int nt, int ld, int T4, const ApplyRow* __restrict__ table,
                                                             const cf* __restrict__ blocks, const cd* x,
                                                             const cd* __restrict__ aux, cd* y, double alpha,
                                                             double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ApplyRow row;
  if (threadIdx.x == 0) row = table[blockIdx.z];
  __syncthreads();
  const int s = blockIdx.x;
  const size_t vs = (size_t)T4 * nt;
  const cd* xs = x + s * vs;
  const cd* as = aux ? aux + s * vs : nullptr;
  const size_t bsz = (size_t)nt * ld;
  const int nterms = row.nterms;  // <= 2 (checked by the launcher's table)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.y * 8 + warp;
  const int np = ld >> 1;
  // (1) this warp's block rows, all loads in flight
  float4 b[2][MAXC];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float4* B = (t < nterms && r < nt)
                          ? reinterpret_cast<const float4*>(blocks + (size_t)row.t[t].block * bsz + (size_t)r * ld)
                          : nullptr;
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      const int k = lane + 32 * c;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (B && k < np) v = __ldg(B + k);
      b[t][c] = v;
    }
  }
  // (2) sign_t (x[in1] + x[in2]) as complex64, padded with zeros to ld
  cf* xin = reinterpret_cast<cf*>(smem_raw);
  for (int t = 0; t < nterms; ++t) {
    const ApplyTerm tm = row.t[t];
    const cd* a = xs + (size_t)tm.in1 * nt;
    const cd* bb = tm.in2 >= 0 ? xs + (size_t)tm.in2 * nt : nullptr;
    for (int k = threadIdx.x; k < ld; k += blockDim.x) {
      cd v = make_double2(0, 0);
      if (k < nt) {
        v = a[k];
        if (bb) v = cadd(v, bb[k]);
        v = cscale(v, tm.sign);
      }
      xin[t * ld + k] = make_float2((float)v.x, (float)v.y);
    }
  }
  __syncthreads();
  if (r >= nt) return;
  // (3) products
  float are = 0.f, aim = 0.f;
  const float4* xv4 = reinterpret_cast<const float4*>(xin);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    if (t >= nterms) break;
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      const int k = lane + 32 * c;
      if (k < np) {
        const float4 v = xv4[t * np + k], bv = b[t][c];
        are = fmaf(bv.x, v.x, are);
        are = fmaf(-bv.y, v.y, are);
        are = fmaf(bv.z, v.z, are);
        are = fmaf(-bv.w, v.w, are);
        aim = fmaf(bv.x, v.y, aim);
        aim = fmaf(bv.y, v.x, aim);
        aim = fmaf(bv.z, v.w, aim);
        aim = fmaf(bv.w, v.z, aim);
      }
    }
  }
  const cf acc = warp_sum_cf(make_float2(are, aim));
  if (lane == 0) {
    cd val = make_double2(acc.x, acc.y);
    for (int e = 0; e < row.nid; ++e) {
      const cd* src = row.id_src[e] == 0 ? xs : as;
      val = cadd(val, cscale(src[(size_t)row.id_trace[e] * nt + r], row.id_sign[e]));
    }
    val = cscale(val, alpha);
    if (beta != 0.0) val = cadd(val, cscale(as[(size_t)row.out * nt + r], beta));
    y[s * vs + (size_t)row.out * nt + r] = val;
  }
}

// FP32 rows of at most two terms, 8 rows per CTA; false when the row length exceeds the register bound
bool launch_apply_f32_rows(int nt, int ld, int T4, const ApplyRow* table, int nrows, const void* blocks, const cd* x,
                           const cd* aux, cd* y, int nsrc, double alpha, double beta, cudaStream_t s,
                           cudaError_t* err) {
  const int np = ld >> 1;
  const size_t smem = 2ull * ld * sizeof(cf);
  dim3 grid(nsrc, (nt + 7) / 8, nrows);
  const cf* B = static_cast<const cf*>(blocks);
  if (np <= 32 * 4) {
    apply_f32_rows_kernel<4><<<grid, 256, smem, s>>>(nt, ld, T4, table, B, x, aux, y, alpha, beta);
  } else if (np <= 32 * 9) {
    apply_f32_rows_kernel<9><<<grid, 256, smem, s>>>(nt, ld, T4, table, B, x, aux, y, alpha, beta);
  } else if (np <= 32 * 18) {
    apply_f32_rows_kernel<18><<<grid, 256, smem, s>>>(nt, ld, T4, table, B, x, aux, y, alpha, beta);
  } else {
    return false;
  }
  *err = cudaGetLastError();
  return true;
}

// ---- conversion of FP64 blocks to the FP32 / double-float layouts -----------
// hi[b][r][k] = fl32(src), lo = fl32(src - hi), rows padded from nt to ld with zeros.
__global__ void split_blocks_kernel(const cd* __restrict__ src, int nt, int ld, size_t nrows_total,
                                    cf* __restrict__ hi, cf* __restrict__ lo) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nrows_total * ld;
       q += (size_t)gridDim.x * blockDim.x) {
    size_t rowi = q / ld;
    int k = (int)(q - rowi * ld);
    cf h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
    if (k < nt) {
      cd v = src[rowi * nt + k];
      h = make_float2((float)v.x, (float)v.y);
      l = make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
    }
    hi[q] = h;
    if (lo) lo[q] = l;
  }
}

cudaError_t launch_apply_mode(int mode, int nt, int ld, int T4, const ApplyRow* table, int nrows,
                              const void* blocks_a, const void* blocks_b, const cd* x, const cd* aux, cd* y,
                              int nsrc, int rows_per_cta, double alpha, double beta, cudaStream_t s) {
  const int elem = mode == kFP32 ? 8 : 16;
  size_t smem = 4ull * ld * elem;
  // sources fastest: the CTAs that read the same block rows for different sources
  // run together, so a batch streams each block from HBM about once (L2 reuse)
  dim3 grid(nsrc, (nt + rows_per_cta - 1) / rows_per_cta, nrows);
  cudaError_t e = cudaSuccess;
  if (mode == kFP64) {
    e = smem_limit_max(reinterpret_cast<const void*>(apply_kernel<kFP64>));
    apply_kernel<kFP64><<<grid, 256, smem, s>>>(nt, ld, T4, table, blocks_a, blocks_b, x, aux, y, rows_per_cta,
                                                alpha, beta);
  } else if (mode == kFP32) {
    e = smem_limit_max(reinterpret_cast<const void*>(apply_kernel<kFP32>));
    apply_kernel<kFP32><<<grid, 256, smem, s>>>(nt, ld, T4, table, blocks_a, blocks_b, x, aux, y, rows_per_cta,
                                                alpha, beta);
  } else {
    e = smem_limit_max(reinterpret_cast<const void*>(apply_kernel<kDF>));
    apply_kernel<kDF><<<grid, 256, smem, s>>>(nt, ld, T4, table, blocks_a, blocks_b, x, aux, y, rows_per_cta,
                                              alpha, beta);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_split_blocks(const cd* src, int nt, int ld, size_t nrows_total, cf* hi, cf* lo, cudaStream_t s) {
  split_blocks_kernel<<<1216, 256, 0, s>>>(src, nt, ld, nrows_total, hi, lo);
  return cudaGetLastError();
}

}  // namespace pt
