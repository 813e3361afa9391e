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

#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

namespace pt {

enum ApplyMode { kFP64 = 0, kFP32 = 1, kDF = 2, kH16 = 3 };

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

// ---- FP32 and double-float applies on inputs converted once ---------------------------
// GB300 issues FP64 instructions at 2 lanes per clock per SM: a warp-wide FP64 instruction
// holds the SM's FP64 pipe for 16 cycles.  Converting every staged input element from
// FP64 in each CTA (35 row tiles per output trace read the same inputs) and running the
// FP64 epilogue of every row on its warp made these HBM-bound applies wait on that pipe.
// Here one pass converts x once per application into xp (DF: float4 (re_hi, im_hi,
// re_lo, im_lo), hi = fl32(v), lo = fl32(v - hi); FP32: float2), rows padded to ld with
// zeros; the apply CTAs stage sign (xp[in1] + xp[in2]) with FP32 (DF: error-free two-sum)
// arithmetic, keep the warp sums in shared memory and let one thread per row add the
// identity terms and the alpha / beta combination in FP64.
__global__ void prep_inputs_kernel(const cd* __restrict__ x, int nt, int ld, int df, void* __restrict__ xp) {
  const size_t v = blockIdx.y;  // source x trace
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ld; k += gridDim.x * blockDim.x) {
    const cd a = k < nt ? x[v * nt + k] : make_double2(0.0, 0.0);
    const float rh = (float)a.x, ih = (float)a.y;
    if (df)
      reinterpret_cast<float4*>(xp)[v * ld + k] =
          make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
    else
      reinterpret_cast<float2*>(xp)[v * ld + k] = make_float2(rh, ih);
  }
}

cudaError_t launch_prep_inputs(const cd* x, int nvec, int nt, int ld, bool df, void* xp, cudaStream_t s) {
  dim3 grid((ld + 255) / 256, nvec);
  prep_inputs_kernel<<<grid, 256, 0, s>>>(x, nt, ld, df ? 1 : 0, xp);
  return cudaGetLastError();
}

// (hi, lo) = a + b for double-float numbers (two-sum of the high parts, low parts folded
// in, renormalised); about 2^-46 relative
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  h = s + e;
  l = e - (h - s);
}

template <int MODE>
__global__ void __launch_bounds__(256) apply_lowp_kernel(int nt, int ld, int T4, const ApplyRow* __restrict__ table,
                                                         const void* __restrict__ blocks_a,
                                                         const void* __restrict__ blocks_b,
                                                         const void* __restrict__ xp, const cd* x,
                                                         const cd* __restrict__ aux, cd* y, int rows_per_cta,
                                                         double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ApplyRow row;
  if (threadIdx.x == 0) row = table[blockIdx.z];
  __syncthreads();
  const int s = blockIdx.x;
  const size_t vs = (size_t)T4 * nt;
  const size_t bsz = (size_t)nt * ld;
  const int nterms = row.nterms;
  const int np = ld >> 1;
  // per-row warp sums after the staged inputs: DF (S_re, C_re, S_im, C_im), FP32 (re, im)
  float4* res = reinterpret_cast<float4*>(smem_raw + (size_t)nterms * ld * (MODE == kDF ? 16 : 8));

  // ---- stage sign_t (xp[in1] + xp[in2]) for every term, FP32 arithmetic only
  for (int t = 0; t < nterms; ++t) {
    const ApplyTerm tm = row.t[t];
    const float sg = (float)tm.sign;  // +-1: exact
    if (MODE == kDF) {
      const float4* a = reinterpret_cast<const float4*>(xp) + ((size_t)s * T4 + tm.in1) * ld;
      const float4* b = tm.in2 >= 0 ? reinterpret_cast<const float4*>(xp) + ((size_t)s * T4 + tm.in2) * ld : nullptr;
      for (int k = threadIdx.x; k < ld; k += blockDim.x) {
        float4 v = a[k];
        if (b) {
          const float4 w = b[k];
          float rh, rl, ih, il;
          df_add(v.x, v.z, w.x, w.z, rh, rl);
          df_add(v.y, v.w, w.y, w.w, ih, il);
          v = make_float4(rh, ih, rl, il);
        }
        reinterpret_cast<float4*>(smem_raw)[t * ld + k] = make_float4(sg * v.x, sg * v.y, sg * v.z, sg * v.w);
      }
    } else {
      const float2* a = reinterpret_cast<const float2*>(xp) + ((size_t)s * T4 + tm.in1) * ld;
      const float2* b = tm.in2 >= 0 ? reinterpret_cast<const float2*>(xp) + ((size_t)s * T4 + tm.in2) * ld : nullptr;
      for (int k = threadIdx.x; k < ld; k += blockDim.x) {
        float2 v = a[k];
        if (b) {
          const float2 w = b[k];
          v = make_float2(v.x + w.x, v.y + w.y);
        }
        reinterpret_cast<float2*>(smem_raw)[t * ld + k] = make_float2(sg * v.x, sg * v.y);
      }
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.y * rows_per_cta;
  for (int rr = warp; rr < rows_per_cta; rr += 8) {
    const int r = r0 + rr;
    if (r >= nt) break;
    if (MODE == kH16) {
      // FP16 block rows, one power-of-two scale per block row: partial sums per term, scaled
      const float4* xin = reinterpret_cast<const float4*>(smem_raw);  // two complex64 per float4
      float are = 0.f, aim = 0.f;
      for (int t = 0; t < nterms; ++t) {
        const int blk = row.t[t].block;
        const uint2* B = reinterpret_cast<const uint2*>(static_cast<const __half2*>(blocks_a) + (size_t)blk * bsz +
                                                        (size_t)r * ld);
        const float sc = __ldg(static_cast<const float*>(blocks_b) + (size_t)blk * nt + r);
        const float4* xv = xin + t * np;
        float tre = 0.f, tim = 0.f;
        for (int k = lane; k < np; k += 32) {
          const uint2 hb = __ldg(B + k);
          const float4 v = xv[k];
          const float2 b0 = __half22float2(*reinterpret_cast<const __half2*>(&hb.x));
          const float2 b1 = __half22float2(*reinterpret_cast<const __half2*>(&hb.y));
          tre = fmaf(b0.x, v.x, tre);
          tre = fmaf(-b0.y, v.y, tre);
          tre = fmaf(b1.x, v.z, tre);
          tre = fmaf(-b1.y, v.w, tre);
          tim = fmaf(b0.x, v.y, tim);
          tim = fmaf(b0.y, v.x, tim);
          tim = fmaf(b1.x, v.w, tim);
          tim = fmaf(b1.y, v.z, tim);
        }
        are = fmaf(tre, sc, are);
        aim = fmaf(tim, sc, aim);
      }
      const cf acc = warp_sum_cf(make_float2(are, aim));
      if (lane == 0) res[rr] = make_float4(acc.x, acc.y, 0.f, 0.f);
    } else if (MODE == kFP32) {
      const float4* xin = reinterpret_cast<const float4*>(smem_raw);  // two complex64 per float4
      float are = 0.f, aim = 0.f;
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
      const cf acc = warp_sum_cf(make_float2(are, aim));
      if (lane == 0) res[rr] = make_float4(acc.x, acc.y, 0.f, 0.f);
    } else {
      const float4* xin = reinterpret_cast<const float4*>(smem_raw);  // (re_hi, im_hi, re_lo, im_lo)
      float Sr = 0.f, Cr = 0.f, Si = 0.f, Ci = 0.f;
      float Sr2 = 0.f, Cr2 = 0.f, Si2 = 0.f, Ci2 = 0.f;
      for (int t = 0; t < nterms; ++t) {
        const size_t off = (size_t)row.t[t].block * bsz + (size_t)r * ld;
        const float4* H = reinterpret_cast<const float4*>(static_cast<const cf*>(blocks_a) + off);
        const float4* Lo = reinterpret_cast<const float4*>(static_cast<const cf*>(blocks_b) + off);
        const float4* xv = xin + t * ld;
        int k = lane;
        // the next pair of columns' block values is loaded while the current pair computes
        float4 nh0, nl0, nh1, nl1;
        if (k + 32 < np) {
          nh0 = __ldg(H + k);
          nl0 = __ldg(Lo + k);
          nh1 = __ldg(H + k + 32);
          nl1 = __ldg(Lo + k + 32);
        }
        for (; k + 32 < np; k += 64) {
          const float4 h0 = nh0, l0 = nl0, h1 = nh1, l1 = nl1;
          if (k + 96 < np) {
            nh0 = __ldg(H + k + 64);
            nl0 = __ldg(Lo + k + 64);
            nh1 = __ldg(H + k + 96);
            nl1 = __ldg(Lo + k + 96);
          }
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
      if (lane == 0) res[rr] = make_float4(Sr, Cr, Si, Ci);
    }
  }
  __syncthreads();
  // ---- FP64 epilogue, one thread per row
  const int rr = threadIdx.x;
  const int r = r0 + rr;
  if (rr < rows_per_cta && r < nt) {
    const float4 v = res[rr];
    cd val = MODE == kDF ? make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w)
                         : make_double2(v.x, v.y);
    const cd* xs = x + s * vs;
    const cd* as = aux ? aux + s * vs : nullptr;
    for (int e = 0; e < row.nid; ++e) {
      const cd* src = row.id_src[e] == 0 ? xs : as;
      val = cadd(val, cscale(src[(size_t)row.id_trace[e] * nt + r], row.id_sign[e]));
    }
    val = cscale(val, alpha);
    if (beta != 0.0) val = cadd(val, cscale(as[(size_t)row.out * nt + r], beta));
    y[s * vs + (size_t)row.out * nt + r] = val;
  }
}

// mode kFP32 (blocks_a: complex64 blocks), kDF (blocks_a / blocks_b: hi / lo complex64) or
// kH16 (blocks_a: FP16 (re, im) pairs, blocks_b: one float scale per block row)
cudaError_t launch_apply_lowp(int mode, int nt, int ld, int T4, const ApplyRow* table, int nrows, const void* blocks_a,
                              const void* blocks_b, const void* xp, const cd* x, const cd* aux, cd* y, int nsrc,
                              int rows_per_cta, double alpha, double beta, cudaStream_t s) {
  if (rows_per_cta > 256) return cudaErrorInvalidValue;
  const int elem = mode == kDF ? 16 : 8;
  const size_t smem = 4ull * ld * elem + (size_t)rows_per_cta * sizeof(float4);
  dim3 grid(nsrc, (nt + rows_per_cta - 1) / rows_per_cta, nrows);
  auto go = [&](auto kern) {
    cudaError_t e = smem_limit_max(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, smem, s>>>(nt, ld, T4, table, blocks_a, blocks_b, xp, x, aux, y, rows_per_cta, alpha, beta);
    return cudaGetLastError();
  };
  if (mode == kDF) return go(apply_lowp_kernel<kDF>);
  if (mode == kH16) return go(apply_lowp_kernel<kH16>);
  return go(apply_lowp_kernel<kFP32>);
}

// FP16 copies of the blocks for the mixed preconditioner: one warp per block row takes the
// row's largest |Re|, |Im| (FP64), picks the power of two 2^p that brings it into
// [2^13, 2^14), stores fl16(2^p b) as (re, im) pairs (rows padded to ld with zeros) and the
// row's scale 2^-p; an entry keeps 11 significant bits unless it is 2^-27 of the row's largest
__global__ void blocks_h16_kernel(const cd* __restrict__ src, int nt, int ld, size_t nrows_total,
                                  __half2* __restrict__ out, float* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const size_t w0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t q = w0; q < nrows_total; q += nw) {
    const cd* row = src + q * nt;
    double m = 0.0;
    for (int k = lane; k < nt; k += 32) m = fmax(m, fmax(fabs(row[k].x), fabs(row[k].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);  // m in [2^(ex-1), 2^ex)
    // the scale 2^-p is stored as a float: p stays in [-127, 126] so that it is a normal
    // number; a row whose largest entry is below 2^-112 then keeps fewer FP16 bits
    const int p = m > 0.0 ? max(-127, min(126, 14 - ex)) : 0;
    const double mult = ldexp(1.0, p);
    for (int k = lane; k < ld; k += 32) {
      float2 v = make_float2(0.f, 0.f);
      if (k < nt) v = make_float2((float)(row[k].x * mult), (float)(row[k].y * mult));
      out[q * ld + k] = __floats2half2_rn(v.x, v.y);
    }
    if (lane == 0) scale[q] = (float)ldexp(1.0, -p);
  }
}

cudaError_t launch_blocks_h16(const cd* src, int nt, int ld, size_t nrows_total, __half2* out, float* scale,
                              cudaStream_t s) {
  blocks_h16_kernel<<<1216, 256, 0, s>>>(src, nt, ld, nrows_total, out, scale);
  return cudaGetLastError();
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

// ---- FP32 D^{-1} in one launch: every sweep step of a cooperative grid ---------
// The steps of a sweep (Section 4.1) form a chain: step s reads the traces that step
// s-1 wrote.  One launch per step pays a launch gap and a full HBM round trip per step
// although the block rows a step multiplies do not depend on the chain.  Here a grid
// that is co-resident (cooperative launch) runs all L-1 steps; warp w of the grid owns
// row rho = w of every step's 4 n_t rows (rho / n_t picks the output trace, rho % n_t
// the row).  As soon as its CTA has finished a step, the warp asks the copy engine for
// its two block rows of the next step (bulk asynchronous copies into shared memory,
// completion on an mbarrier): the next step's HBM stream runs during the grid barrier
// and the staging of the new inputs, and it does not hold the SM's load slots, which
// register loads of 141 KB per SM would exhaust.  The grid barrier is one arrival
// counter, zeroed before the launch; every wait is bounded (kErrTimeout, then the grid
// returns, after its own copies have landed).
// Layout the host checks before it takes this path: rows 2g and 2g+1 of a step (g = 0:
// the down-going pair, g = 1: the up-going pair) have the same terms (input trace, sign)
// and differ only in their blocks; a term has one input trace; identities read the
// auxiliary vector; alpha = 1, beta = 0; every row has a warp (4 n_t <= 16 x grid).
constexpr int kSweepThreads = 512;
constexpr int kSweepWarps = kSweepThreads / 32;

__device__ __forceinline__ unsigned long long sweep_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned sweep_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void sweep_arrive(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ uint32_t sweep_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// wait for phase `parity` of the copy mbarrier, at most 1 s; false (and kErrTimeout) on expiry
__device__ __forceinline__ bool sweep_mb_wait(uint64_t* mb, int parity, int* status) {
  const unsigned long long t0 = sweep_timer();
  for (long long it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sweep_saddr(mb)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && sweep_timer() - t0 > 1000000000ull) break;
  }
  atomicOr(status, kErrTimeout);
  return false;
}

// H16: FP16 block rows ((re, im) pairs) with one float scale per block row (bscale), half
// the bytes per step; products per term in FP32, scaled, then summed
template <int MAXC, bool H16>
__global__ void __launch_bounds__(kSweepThreads, 1)
    sweep_f32_kernel(int nt, int ld, int T4, int nsteps, const ApplyRow* __restrict__ table,
                     const void* __restrict__ blocks, const float* __restrict__ bscale, const cd* __restrict__ aux,
                     cd* y, cf* y32, int S, unsigned* bar, int* status) {
  using E = typename std::conditional<H16, __half2, cf>::type;  // one complex block entry
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int abort_flag;
  // [step table: 4 nsteps rows][block rows: warp x term x ld][inputs: S x (2 g + t) x ld]
  // [row sums: warp x S][one mbarrier per warp]
  ApplyRow* tab = reinterpret_cast<ApplyRow*>(smem_raw);
  E* buf = reinterpret_cast<E*>(smem_raw + (size_t)4 * nsteps * sizeof(ApplyRow));
  cf* xin = reinterpret_cast<cf*>(buf + (size_t)kSweepWarps * 2 * ld);
  cf* sums = xin + (size_t)S * 4 * ld;
  uint64_t* mbs = reinterpret_cast<uint64_t*>(sums + (((size_t)kSweepWarps * S + 1) & ~(size_t)1));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * kSweepWarps + warp;
  const int Rn = 4 * nt;
  const bool own = gw < Rn;
  const int qt = own ? gw / nt : 0, r = own ? gw % nt : 0, g = qt >> 1;
  const size_t vs = (size_t)T4 * nt;
  const int np = ld >> 1;
  // the pairs of output traces this CTA's rows touch
  const int r_lo = blockIdx.x * kSweepWarps, r_hi = min(r_lo + kSweepWarps, Rn) - 1;
  const int g_lo = r_lo / (2 * nt), g_hi = r_hi / (2 * nt);
  const int ng = g_hi - g_lo + 1;
  // output thread: (row w of this CTA, source q), w S + q = threadIdx.x < kSweepWarps S.  The
  // FP64 part of a row (the identity terms) runs here, on few warps: one warp-wide FP64
  // instruction occupies the SM's FP64 pipe for 16 cycles on this part.
  const bool outer = threadIdx.x < kSweepWarps * S;
  const int ow = outer ? threadIdx.x / S : 0, oq = threadIdx.x - ow * S;
  const int orow = r_lo + ow;
  const bool oown = outer && orow < Rn;
  const int oqt = oown ? orow / nt : 0, or_ = oown ? orow % nt : 0;
  {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(table);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(tab);
    const int nw = (int)(4 * nsteps * sizeof(ApplyRow) / 8);
    for (int i = threadIdx.x; i < nw; i += kSweepThreads) dst[i] = src[i];
  }
  uint64_t* mb = mbs + warp;  // this warp's copies
  if (threadIdx.x == 0) abort_flag = 0;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sweep_saddr(mb)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // lane 0 of every warp: its block rows of step st by the copy engine, on its own mbarrier
  // (one arrival per phase, with the bytes it asked for), so that each warp starts its
  // products as soon as its rows have landed; output threads: their identity terms
  double2 a[2];
  float sc_next[2] = {1.f, 1.f};  // H16: the row scales of the warp's next block rows
  auto issue = [&](int st) {
    const ApplyRow* row = tab + 4 * st + qt;
    if (lane == 0) {
      const int nterms = own ? row->nterms : 0;
      const uint32_t bytes = (uint32_t)(nterms * ld * sizeof(E));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic reads of the buffer first
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sweep_saddr(mb)), "r"(bytes)
                   : "memory");
      for (int t = 0; t < nterms; ++t)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sweep_saddr(buf + (size_t)(warp * 2 + t) * ld)),
            "l"(static_cast<const E*>(blocks) + ((size_t)row->t[t].block * nt + r) * ld),
            "r"((uint32_t)(ld * sizeof(E))), "r"(sweep_saddr(mb))
            : "memory");
    }
    if (H16) {
      const int nterms = own ? row->nterms : 0;
#pragma unroll
      for (int t = 0; t < 2; ++t) sc_next[t] = t < nterms ? __ldg(bscale + (size_t)row->t[t].block * nt + r) : 0.f;
    }
    const ApplyRow* orw = tab + 4 * st + oqt;
    const int nid = orw->nid;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      double2 v = make_double2(0.0, 0.0);
      if (oown && e < nid) v = __ldg(aux + (size_t)oq * vs + (size_t)orw->id_trace[e] * nt + or_);
      a[e] = v;
    }
  };

  issue(0);
  for (int s = 0; s < nsteps; ++s) {
    const ApplyRow* rows = tab + 4 * s;
    if (s > 0) {  // grid barrier: every output of step s-1 is written
      if (threadIdx.x == 0) {
        const unsigned target = (unsigned)s * gridDim.x;
        const unsigned long long t0 = sweep_timer();
        for (long long it = 0;; ++it) {
          if (sweep_ld_acquire(bar) >= target) break;
          if ((it & 255) == 255 && sweep_timer() - t0 > 1000000000ull) {
            atomicOr(status, kErrTimeout);
            abort_flag = 1;
            break;
          }
        }
      }
      __syncthreads();
      if (abort_flag) {  // let this step's copies land before the shared memory goes away
        sweep_mb_wait(mb, s & 1, status);
        return;
      }
    }
    // (1) stage sign_t y32[in_t] of the touched pairs (the complex64 copies of the traces that
    //     the previous steps wrote, read from L2), zero-padded to ld: slot j = 2 (g - g_lo) + t
    //     of source q; two (q, j) pairs at a time, a thread's loads before its stores
    {
      const int nslot = 2 * ng, sh = ng == 2 ? 2 : 1, npair = S * nslot;
      for (int p0 = 0; p0 < npair; p0 += 2) {
        cf v[2][2];
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int p = p0 + pp, jj = p & (nslot - 1), q = p >> sh, t = jj & 1;
          const ApplyRow* pr = rows + 2 * (g_lo + (jj >> 1));
          const bool live = p < npair && t < pr->nterms;
          const cf* src = y32 + (size_t)q * vs + (size_t)(live ? pr->t[t].in1 : 0) * nt;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int k = threadIdx.x + u * kSweepThreads;
            v[pp][u] = (live && k < nt) ? __ldcg(src + k) : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int p = p0 + pp, jj = p & (nslot - 1), q = p >> sh, t = jj & 1;
          if (p < npair) {
            const ApplyRow* pr = rows + 2 * (g_lo + (jj >> 1));
            const float sg = t < pr->nterms ? (float)pr->t[t].sign : 0.f;
            cf* dst = xin + ((size_t)q * 4 + 2 * g_lo + jj) * ld;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int k = threadIdx.x + u * kSweepThreads;
              if (k < ld) dst[k] = make_float2(sg * v[pp][u].x, sg * v[pp][u].y);
            }
          }
        }
      }
    }
    __syncthreads();
    // (2) this warp's block rows landed, (3) its row products (FP32), one sum per source
    //     into shared memory
    const bool ok = sweep_mb_wait(mb, s & 1, status);
    const float sc0 = sc_next[0], sc1 = sc_next[1];
    if (own && ok) {
      const int nterms = rows[qt].nterms;
      for (int q = 0; q < S; ++q) {
        float are = 0.f, aim = 0.f;
        const float4* xv4 = reinterpret_cast<const float4*>(xin + (size_t)q * 4 * ld);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (H16 && t < nterms) {
            const uint2* bh = reinterpret_cast<const uint2*>(buf + (size_t)(warp * 2 + t) * ld);
            float tre = 0.f, tim = 0.f;
#pragma unroll
            for (int c = 0; c < MAXC; ++c) {
              const int k = lane + 32 * c;
              if (k < np) {
                const float4 v = xv4[(2 * g + t) * np + k];
                const uint2 hb = bh[k];
                const float2 b0 = __half22float2(*reinterpret_cast<const __half2*>(&hb.x));
                const float2 b1 = __half22float2(*reinterpret_cast<const __half2*>(&hb.y));
                tre = fmaf(b0.x, v.x, tre);
                tre = fmaf(-b0.y, v.y, tre);
                tre = fmaf(b1.x, v.z, tre);
                tre = fmaf(-b1.y, v.w, tre);
                tim = fmaf(b0.x, v.y, tim);
                tim = fmaf(b0.y, v.x, tim);
                tim = fmaf(b1.x, v.w, tim);
                tim = fmaf(b1.y, v.z, tim);
              }
            }
            const float sct = t == 0 ? sc0 : sc1;
            are = fmaf(tre, sct, are);
            aim = fmaf(tim, sct, aim);
          } else if (!H16 && t < nterms) {
            const float4* bv4 = reinterpret_cast<const float4*>(reinterpret_cast<const cf*>(buf) + (size_t)(warp * 2 + t) * ld);
#pragma unroll
            for (int c = 0; c < MAXC; ++c) {
              const int k = lane + 32 * c;
              if (k < np) {
                const float4 v = xv4[(2 * g + t) * np + k], bv = bv4[k];
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
        }
        const cf acc = warp_sum_cf(make_float2(are, aim));
        if (lane == 0) sums[warp * S + q] = acc;
      }
    }
    if (__syncthreads_or(!ok)) return;
    // (4) outputs: y = sum + identity terms (FP64), and its complex64 copy for the next steps
    if (oown) {
      const ApplyRow* row = rows + oqt;
      const cf acc = sums[ow * S + oq];
      cd val = make_double2(acc.x, acc.y);
      const int nid = row->nid;
#pragma unroll
      for (int e = 0; e < 2; ++e)
        if (e < nid) val = cadd(val, cscale(a[e], row->id_sign[e]));
      const size_t o = (size_t)oq * vs + (size_t)row->out * nt + or_;
      y[o] = val;
      y32[o] = make_float2((float)val.x, (float)val.y);
    }
    // (5) arrive (a release: it waits for this CTA's stores), then the next step's copies,
    //     which must not be in flight while the release drains the SM's memory operations
    __syncthreads();
    if (s + 1 < nsteps) {
      if (threadIdx.x == 0) sweep_arrive(bar);
      __syncthreads();
      issue(s + 1);
    }
  }
}

size_t sweep_f32_smem(int ld, int S, int nsteps, bool h16) {
  return (size_t)4 * nsteps * sizeof(ApplyRow) + (size_t)kSweepWarps * 2 * ld * (h16 ? sizeof(__half2) : sizeof(cf)) +
         (size_t)S * 4 * ld * sizeof(cf) + ((((size_t)kSweepWarps * S + 1) & ~(size_t)1) * sizeof(cf)) +
         kSweepWarps * sizeof(uint64_t);
}

// D^{-1} of the mixed preconditioner in one cooperative launch, with complex64 blocks or, when
// bscale is given, FP16 blocks and their row scales; y32 (S x T4 x n_t complex64) is scratch.
// False (nothing launched) when the shape is outside the kernel's bounds (register tile,
// shared memory, one warp per row of a step on a co-resident grid).
bool launch_sweep_f32(int nt, int ld, int T4, int nsteps, const ApplyRow* table, const void* blocks,
                      const float* bscale, const cd* aux, cd* y, cf* y32, int S, unsigned* bar, int* status,
                      cudaStream_t s, cudaError_t* err) {
  const int np = ld >> 1;
  const bool h16 = bscale != nullptr;
  if (nsteps < 1 || nsteps > 64 || S < 1 || S > 32 || ld > 2 * kSweepThreads) return false;
  const void* fn;
  if (np <= 32 * 4) fn = h16 ? reinterpret_cast<const void*>(sweep_f32_kernel<4, true>)
                             : reinterpret_cast<const void*>(sweep_f32_kernel<4, false>);
  else if (np <= 32 * 9) fn = h16 ? reinterpret_cast<const void*>(sweep_f32_kernel<9, true>)
                                  : reinterpret_cast<const void*>(sweep_f32_kernel<9, false>);
  else return false;
  const size_t smem = sweep_f32_smem(ld, S, nsteps, h16);
  int dev = 0, sms = 0, occ = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && smem + 64 > (size_t)optin) return false;
  if (e == cudaSuccess) e = smem_limit_max(fn);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSweepThreads, smem);
  if (e != cudaSuccess) {
    *err = e;
    return true;
  }
  const int R = 4 * nt;
  const int G = (R + kSweepWarps - 1) / kSweepWarps;
  if (occ < 1 || G > sms * occ) return false;
  e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    const ApplyRow* tb = table;
    const void* bl = blocks;
    const float* bs = bscale;
    void* args[] = {(void*)&nt, (void*)&ld, (void*)&T4, (void*)&nsteps, (void*)&tb, (void*)&bl, (void*)&bs,
                    (void*)&aux, (void*)&y, (void*)&y32, (void*)&S, (void*)&bar, (void*)&status};
    e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kSweepThreads), args, smem, s);
  }
  *err = e;
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
