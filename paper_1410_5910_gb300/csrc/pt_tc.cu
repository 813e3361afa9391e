// Batched block applies on the tensor cores (tcgen05, TMEM, TMA).
//
// With S sources the products of an operator table (Definition 9 after P,
// its coupling R, or one sweep step of Section 4.1) are dense contractions.
// Complex arithmetic is carried as real blocks: a block B = Br + i Bi is
// stored as the K-concatenation A = [Br Bi] (n_t x 2 n_t) and a term's input
// X (n_t x S complex, sign folded in) as the K-major operand
//     Xop^T = [[Xr^T, -Xi^T], [Xi^T, Xr^T]]   (2S x 2 n_t),
// so that A Xop = [Re(B X) | Im(B X)] (n_t x 2S).  The terms of an output
// trace are consecutive K ranges of one accumulator.
//
// Precision: FP16 operands with power-of-two scales (one for all blocks, one
// per source), FP32 accumulation in tensor memory.  One pass (A_hi X_hi) for
// the preconditioner, or the three-pass split A_hi X_hi + A_hi X_lo + A_lo X_hi
// (hi = fl16(v), lo = fl16(v - hi)) for the GMRES matvec.
//
// Kernel structure (one CTA per 128 x BN output tile, 128 threads): thread 0
// issues TMA loads into a 4-stage shared-memory ring (128-byte swizzle),
// thread 32 issues tcgen05.mma (M = 128, N = BN, K = 16) into a TMEM
// accumulator, all four warps read the accumulator back with tcgen05.ld.
// Every mbarrier wait gives up after 2 s of wall-clock time, records
// kErrTimeout and lets the kernel finish (TMEM is always released).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "pt_common.cuh"

namespace pt {

constexpr int kTcBM = 128, kTcBK = 64, kTcStages = 4;


__device__ __forceinline__ uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long tc_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void tc_mb_init(uint64_t* b, int c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_saddr(b)), "r"(c));
}
__device__ __forceinline__ void tc_mb_expect(uint64_t* b, int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_saddr(b)), "r"(bytes) : "memory");
}
// bounded wait: false after 2 s (status gets kErrTimeout)
__device__ __forceinline__ bool tc_mb_wait(uint64_t* b, int phase, int* status) {
  const unsigned long long t0 = tc_timer();
  for (long long it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc_saddr(b)), "r"(phase)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && tc_timer() - t0 > 2000000000ull) break;
  }
  atomicOr(status, kErrTimeout);
  return false;
}
__device__ __forceinline__ void tc_tma_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(tc_saddr(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(tc_saddr(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t a) {
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <int BN>
__global__ void __launch_bounds__(128) tc_apply_kernel(
    const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
    const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
    const TcRow* __restrict__ rows, int nt, int T4, int S, int npass, const float* __restrict__ inv_scale,
    const cd* x, const cd* __restrict__ aux, cd* y, double alpha, double beta, int* status) {
  constexpr int A_BYTES = kTcBM * kTcBK * 2, B_BYTES = BN * kTcBK * 2, STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t kIdesc =
      (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ TcRow row;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * BN;
  if (threadIdx.x == 0) {
    row = rows[blockIdx.z];
    for (int s = 0; s < kTcStages; ++s) {
      tc_mb_init(&full[s], 1);
      tc_mb_init(&empty[s], 1);
    }
    tc_mb_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&tmem_base)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int nkb = (2 * nt + kTcBK - 1) / kTcBK;
  const int total = npass * row.nterms * nkb;
  if (warp == 0 && lane == 0) {
    for (int it = 0; it < total; ++it) {
      const int s = it % kTcStages, u = it / kTcStages;
      if (it >= kTcStages && !tc_mb_wait(&empty[s], (u & 1) ^ 1, status)) break;
      const int pass = it / (row.nterms * nkb);
      const int rem = it - pass * row.nterms * nkb;
      const int t = rem / nkb, kb = rem - (rem / nkb) * nkb;
      const CUtensorMap* ta = pass == 2 ? &tmAlo : &tmAhi;
      const CUtensorMap* tb = pass == 1 ? &tmBlo : &tmBhi;
      tc_mb_expect(&full[s], STAGE);
      tc_tma_2d(smem + s * STAGE, ta, kb * kTcBK, row.t[t].a_row0 + m0, &full[s]);
      tc_tma_2d(smem + s * STAGE + A_BYTES, tb, kb * kTcBK, row.t[t].key * 2 * S + n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    for (int it = 0; it < total; ++it) {
      const int s = it % kTcStages, u = it / kTcStages;
      if (!tc_mb_wait(&full[s], u & 1, status)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = tc_saddr(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        const uint64_t ad = tc_sdesc(a0 + kk * 32), bd = tc_sdesc(b0 + kk * 32);
        const uint32_t acc = (it | kk) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_saddr(&empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_saddr(&done))
                 : "memory");
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, tc_mb_wait(&done, 0, status));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int r = m0 + warp * 32 + lane;
  const size_t vs = (size_t)T4 * nt;
  if (ok) {
    for (int cc = 0; cc < BN / 32; ++cc) {
      uint32_t v[32];
      if (total > 0) {
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + cc * 32;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0u;  // no block term: only the identity terms remain
      }
      if (r < nt) {
        // FP32 arithmetic (the products carry ~1e-5 at best): GB300's FP64 pipe takes 16 cycles per
        // warp instruction, and an FP64 epilogue over 128 x BN outputs outlasted the MMAs of a sweep
        // step; FP64 only for the loads, one conversion each, and the store
        const float fa = (float)alpha, fb = (float)beta;
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + cc * 32 + j;
          if (col >= 2 * S) break;
          const int s = col < S ? col : col - S;
          const int im = col >= S ? 1 : 0;
          float val = __uint_as_float(v[j]) * inv_scale[s];
          const cd* xs = x + (size_t)s * vs;
          const cd* as = aux ? aux + (size_t)s * vs : nullptr;
          for (int e = 0; e < row.nid; ++e) {
            const cd* src = row.id_src[e] == 0 ? xs : as;
            const double q = reinterpret_cast<const double*>(src + (size_t)row.id_trace[e] * nt + r)[im];
            val += (row.id_sign[e] > 0.0 ? 1.0f : -1.0f) * __double2float_rn(q);
          }
          val *= fa;
          if (beta != 0.0) val += fb * __double2float_rn(reinterpret_cast<const double*>(as + (size_t)row.out * nt + r)[im]);
          reinterpret_cast<double*>(y + (size_t)s * vs + (size_t)row.out * nt + r)[im] = (double)val;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// ---- operand preparation --------------------------------------------------------
// Per-source scale 2^e with max |x_s| * 2^e in [2^9, 2^10) (64x FP16 headroom for sums and sweep growth):
// scale[s] = 2^e, inv[s] = 2^-(e + eA).
__global__ void tc_source_scale_kernel(const cd* __restrict__ x, size_t per_src, int eA, float* __restrict__ scale,
                                       float* __restrict__ inv) {
  const int s = blockIdx.x;
  double m = 0.0;
  for (size_t k = threadIdx.x; k < per_src; k += blockDim.x) {
    const cd v = x[(size_t)s * per_src + k];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    int e = 0;
    if (mm > 0) {
      int ex;
      frexp(mm, &ex);  // mm = f 2^ex, f in [0.5, 1)
      e = 10 - ex;
    }
    e = max(-120, min(120, e));
    scale[s] = ldexpf(1.0f, e);
    inv[s] = (float)ldexp(1.0, -(e + eA));
  }
}

// Staged operand of key k: rows [k * 2S, (k + 1) * 2S) of the stacked tensor, ld halves per row.
// row s: [Re X_s | -Im X_s], row S + s: [Im X_s | Re X_s], X_s = sign (x_s[in1] + x_s[in2]) * scale[s].
__global__ void tc_stage_kernel(const TcKey* __restrict__ keys, int nkeys, const cd* __restrict__ x, int nt, int T4,
                                int S, int ld, const float* __restrict__ scale, __half* __restrict__ hi,
                                __half* __restrict__ lo) {
  const int half_ld = ld / 2;  // >= nt; entries j in [nt, half_ld) are the zero padding of each half row
  const size_t total = (size_t)nkeys * S * half_ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / ((size_t)S * half_ld));
    const size_t rem = q - (size_t)k * S * half_ld;
    const int s = (int)(rem / half_ld), j = (int)(rem - (size_t)s * half_ld);
    if (j >= nt) {
      // padding: columns 2 nt .. ld of both rows of this source (j - nt < ld/2 - nt covers them twice over)
      const size_t rr = ((size_t)k * 2 * S + s) * ld, ri = ((size_t)k * 2 * S + S + s) * ld;
      const int c = 2 * nt + 2 * (j - nt);
      for (int d = 0; d < 2; ++d)
        if (c + d < ld) {
          hi[rr + c + d] = __float2half(0.f);
          hi[ri + c + d] = __float2half(0.f);
          if (lo) { lo[rr + c + d] = __float2half(0.f); lo[ri + c + d] = __float2half(0.f); }
        }
      continue;
    }
    const TcKey key = keys[k];
    const cd* xs = x + (size_t)s * T4 * nt;
    // FP32 arithmetic: the hi / lo split keeps 22 bits (FP32 has 24); FP64 only for the loads
    const cd a = xs[(size_t)key.in1 * nt + j];
    float vr = __double2float_rn(a.x), vi = __double2float_rn(a.y);
    if (key.in2 >= 0) {
      const cd b = xs[(size_t)key.in2 * nt + j];
      vr += __double2float_rn(b.x);
      vi += __double2float_rn(b.y);
    }
    const float sc = (key.sign > 0.0 ? 1.0f : -1.0f) * scale[s];
    const float re = vr * sc, imv = vi * sc;
    const __half rh = __float2half_rn(re), ih = __float2half_rn(imv);
    const __half mih = __hneg(ih);
    const size_t rr = ((size_t)k * 2 * S + s) * ld, ri = ((size_t)k * 2 * S + S + s) * ld;
    hi[rr + j] = rh;
    hi[rr + nt + j] = mih;
    hi[ri + j] = ih;
    hi[ri + nt + j] = rh;
    if (lo) {
      const __half rl = __float2half_rn(re - __half2float(rh));
      const __half il = __float2half_rn(imv - __half2float(ih));
      lo[rr + j] = rl;
      lo[rr + nt + j] = __hneg(il);
      lo[ri + j] = il;
      lo[ri + nt + j] = rl;
    }
  }
}

// Blocks to FP16 [Br Bi] rows with the global scale 2^eA (offline); padding columns 2 nt .. ld are zero.
__global__ void tc_blocks_kernel(const cd* __restrict__ blocks, size_t nrows, int nt, int ld, double scale,
                                 __half* __restrict__ hi, __half* __restrict__ lo) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nrows * nt; q += (size_t)gridDim.x * blockDim.x) {
    const size_t r = q / nt;
    const int j = (int)(q - r * nt);
    for (int c = 2 * nt + j; c < ld; c += nt) {
      hi[r * ld + c] = __float2half(0.f);
      lo[r * ld + c] = __float2half(0.f);
    }
    const cd v = blocks[q];
    const double re = v.x * scale, im = v.y * scale;
    const __half rh = __double2half(re), ih = __double2half(im);
    hi[r * ld + j] = rh;
    hi[r * ld + nt + j] = ih;
    lo[r * ld + j] = __double2half(re - (double)__half2float(rh));
    lo[r * ld + nt + j] = __double2half(im - (double)__half2float(ih));
  }
}

__global__ void max_abs_kernel(const cd* __restrict__ v, size_t n, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fmax(fabs(v[q].x), fabs(v[q].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));  // m >= 0: bit order = value order
}

// ---- Exact split products for the explicit residual of a restart (tensor cores) -----------
// The error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) for matrix products: each
// operand row is scaled by a power of two into (-1, 1) and cut into kOzP slices of kOzW bits,
//     v = 2^e sum_i a_i 2^{-7 i},   a_1 = rint(2^7 R_0), a_{i+1} = rint(2^7 R_i),
//     R_0 = v 2^-e, R_i = 2^7 R_{i-1} - a_i,
// with integer slices |a_1| <= 128, |a_i| <= 64 (i > 1), held exactly in FP16.  A product of two
// slices is an integer below 2^14, and a sum of 512 of them at one level i + j stays below 2^24,
// so the tensor cores' FP32 accumulation of one 512-long K segment is exact; the segments are
// added into double-float accumulators with power-of-two weights 2^{-7 (i + j)}.  Slice pairs
// with i + j > kOzLevels + 1 (1-based) are dropped: the product keeps about 35 bits, relative to
// the largest entry of the block row times the largest entry of the source's vector (~1e-10
// on the blocks of the jump system, against ~1e-14 for double-float and 1e-5 for the
// three-pass FP16 matvec).
constexpr int kOzW = 7;
constexpr int kOzP = 5;          // slices per operand
constexpr int kOzLevels = 5;     // 0-based levels i + j = 0 .. 4: 15 slice pairs
constexpr int kOzBN = 48;        // output columns (real parts / imaginary parts of sources) per CTA
constexpr int kOzStages = 2;
constexpr int kOzSegBlocks = 8;  // K blocks (of 64) per exact segment
constexpr int kOzThreads = 192;  // warp 0: TMA, warp 1: MMA, warps 2-5: accumulators and epilogue

// Offline: block rows [Br Bi] (FP64) to kOzP FP16 slice arrays (slice-major, ld halves per row,
// padding zero) and the row exponents e with max |row| < 2^e; one warp per block row.
__global__ void oz_blocks_kernel(const cd* __restrict__ blocks, size_t nrows, int nt, int ld,
                                 __half* __restrict__ out, int* __restrict__ ex) {
  const int lane = threadIdx.x & 31;
  const size_t w0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t q = w0; q < nrows; q += nw) {
    const cd* row = blocks + q * nt;
    double m = 0.0;
    for (int k = lane; k < nt; k += 32) m = fmax(m, fmax(fabs(row[k].x), fabs(row[k].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    if (m > 0.0) frexp(m, &e);  // m in [2^(e-1), 2^e)
    for (int k = lane; k < ld; k += 32) {
      double v = 0.0;
      if (k < nt) v = row[k].x;
      else if (k < 2 * nt) v = row[k - nt].y;
      double R = ldexp(v, -e);
#pragma unroll
      for (int i = 0; i < kOzP; ++i) {
        R *= 128.0;
        const double a = rint(R);
        R -= a;
        out[(size_t)i * nrows * ld + q * ld + k] = __double2half(a);
      }
    }
    if (lane == 0) ex[q] = e;
  }
}

// Per-source exponent f with max |x_s| < 2^(f - 1): staged inputs sum two traces at most.
__global__ void oz_source_exp_kernel(const cd* __restrict__ x, size_t per_src, int* __restrict__ fexp) {
  const int s = blockIdx.x;
  double m = 0.0;
  for (size_t k = threadIdx.x; k < per_src; k += blockDim.x) {
    const cd v = x[(size_t)s * per_src + k];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    int e = 0;
    if (mm > 0.0) frexp(mm, &e);
    fexp[s] = mm > 0.0 ? e + 1 : 0;
  }
}

// Staged input slices of key k for source s (rows k 2S + s: [Re X | -Im X], k 2S + S + s:
// [Im X | Re X]) in kOzP slice-major arrays of slice_rows rows, X = sign (x[in1] + x[in2]).
__global__ void oz_stage_kernel(const TcKey* __restrict__ keys, int nkeys, const cd* __restrict__ x, int nt, int T4,
                                int S, int ld, const int* __restrict__ fexp, size_t slice_rows,
                                __half* __restrict__ out) {
  const int half_ld = ld / 2;
  const size_t total = (size_t)nkeys * S * half_ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / ((size_t)S * half_ld));
    const size_t rem = q - (size_t)k * S * half_ld;
    const int s = (int)(rem / half_ld), j = (int)(rem - (size_t)s * half_ld);
    const size_t rr = ((size_t)k * 2 * S + s) * ld, ri = ((size_t)k * 2 * S + S + s) * ld;
    if (j >= nt) {  // padding columns 2 nt .. ld of both rows, every slice
      const int c = 2 * nt + 2 * (j - nt);
      for (int i = 0; i < kOzP; ++i)
        for (int d = 0; d < 2; ++d)
          if (c + d < ld) {
            out[(size_t)i * slice_rows * ld + rr + c + d] = __float2half(0.f);
            out[(size_t)i * slice_rows * ld + ri + c + d] = __float2half(0.f);
          }
      continue;
    }
    const TcKey key = keys[k];
    const cd* xs = x + (size_t)s * T4 * nt;
    cd v = xs[(size_t)key.in1 * nt + j];
    if (key.in2 >= 0) v = cadd(v, xs[(size_t)key.in2 * nt + j]);
    const int f = fexp[s];
    double Rr = ldexp(key.sign * v.x, -f), Ri = ldexp(key.sign * v.y, -f);
#pragma unroll
    for (int i = 0; i < kOzP; ++i) {
      Rr *= 128.0;
      Ri *= 128.0;
      const double ar = rint(Rr), ai = rint(Ri);
      Rr -= ar;
      Ri -= ai;
      __half* o = out + (size_t)i * slice_rows * ld;
      const __half hr = __double2half(ar), hi = __double2half(ai), mhi = __double2half(-ai);
      o[rr + j] = hr;
      o[rr + nt + j] = mhi;
      o[ri + j] = hi;
      o[ri + nt + j] = hr;
    }
  }
}

// (hi, lo) += v for an FP32 v (Knuth's two-sum; the error term collected in lo)
__device__ __forceinline__ void oz_acc(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ float oz_pow2(int E) { return E < -126 ? 0.f : ldexpf(1.0f, E); }

// One CTA per 128 x kOzBN output tile of one output trace (grid z) of the operator table: y =
// alpha (sum of the terms' block products + identity terms) + beta aux, the block products by
// the split products above.  Two shared-memory stages, each holding the kOzP slices of a
// 128 x 64 block-row tile and of a kOzBN x 64 input tile (128-byte swizzle); five FP32
// accumulators (levels) of kOzBN columns in tensor memory, reset every segment.
__global__ void __launch_bounds__(kOzThreads, 1) oz_apply_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, const TcRow* __restrict__ rows,
    int nt, int T4, int S, int a_slice_rows, int x_slice_rows, const int* __restrict__ aexp,
    const int* __restrict__ fexp, const cd* x, const cd* __restrict__ aux, cd* y, double alpha, double beta,
    int* status) {
  constexpr int A_BYTES = kTcBM * kTcBK * 2, X_BYTES = kOzBN * kTcBK * 2;
  constexpr int STAGE = kOzP * (A_BYTES + X_BYTES);
  constexpr uint32_t kIdesc =
      (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kOzBN >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
  extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kOzStages], empty[kOzStages], seg_full, seg_free, done;
  __shared__ uint32_t tmem_base;
  __shared__ TcRow row;
  __shared__ int abort_flag, issued, consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * kOzBN;
  if (threadIdx.x == 0) {
    row = rows[blockIdx.z];
    for (int s = 0; s < kOzStages; ++s) {
      tc_mb_init(&full[s], 1);
      tc_mb_init(&empty[s], 1);
    }
    tc_mb_init(&seg_full, 1);
    tc_mb_init(&seg_free, 4);
    tc_mb_init(&done, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int nkb = (2 * nt + kTcBK - 1) / kTcBK;
  const int segs_per_term = (nkb + kOzSegBlocks - 1) / kOzSegBlocks;
  const int total = row.nterms * nkb;
  const int nseg = row.nterms * segs_per_term;

  if (warp == 0 && lane == 0) {  // ---- TMA producer
    int it = 0;
    for (; it < total; ++it) {
      const int s = it % kOzStages, u = it / kOzStages;
      if (it >= kOzStages && !tc_mb_wait(&empty[s], (u & 1) ^ 1, status)) { atomicExch(&abort_flag, 1); break; }
      if (*(volatile int*)&abort_flag) break;
      const int t = it / nkb, kb = it - t * nkb;
      unsigned char* st = smem + s * STAGE;
      tc_mb_expect(&full[s], STAGE);
      for (int i = 0; i < kOzP; ++i)
        tc_tma_2d(st + i * A_BYTES, &tmA, kb * kTcBK, i * a_slice_rows + row.t[t].a_row0 + m0, &full[s]);
      for (int j = 0; j < kOzP; ++j)
        tc_tma_2d(st + kOzP * A_BYTES + j * X_BYTES, &tmX, kb * kTcBK, j * x_slice_rows + row.t[t].key * 2 * S + n0,
                  &full[s]);
    }
    issued = it;
  } else if (warp == 1 && lane == 0) {  // ---- MMA issuer
    int it = 0, seg = 0;
    for (; it < total; ++it) {
      const int s = it % kOzStages, u = it / kOzStages;
      const int t = it / nkb, kb = it - t * nkb;
      const bool first = kb % kOzSegBlocks == 0;
      const bool last = kb % kOzSegBlocks == kOzSegBlocks - 1 || kb == nkb - 1;
      // the accumulators of the previous segment must have been read before they are reset
      if (first && seg > 0 && !tc_mb_wait(&seg_free, (seg - 1) & 1, status)) { atomicExch(&abort_flag, 1); break; }
      if (!tc_mb_wait(&full[s], u & 1, status)) { atomicExch(&abort_flag, 1); break; }
      if (*(volatile int*)&abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = tc_saddr(smem + s * STAGE), x0 = a0 + kOzP * A_BYTES;
      uint32_t fresh = first ? 0x1Fu : 0u;  // levels not yet written in this segment
#pragma unroll 1
      for (int i = 0; i < kOzP; ++i) {
#pragma unroll 1
        for (int j = 0; i + j < kOzLevels; ++j) {
          const int l = i + j;
          const uint32_t d = tmem + (uint32_t)(l * 64);
#pragma unroll
          for (int kk = 0; kk < kTcBK / 16; ++kk) {
            const uint64_t ad = tc_sdesc(a0 + i * A_BYTES + kk * 32), bd = tc_sdesc(x0 + j * X_BYTES + kk * 32);
            const uint32_t acc = (fresh >> l) & 1u ? 0u : 1u;
            fresh &= ~(1u << l);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_saddr(&empty[s]))
                   : "memory");
      if (last) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc_saddr(&seg_full))
                     : "memory");
        ++seg;
      }
    }
    consumed = it;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_saddr(&done))
                 : "memory");
  } else if (warp >= 2) {  // ---- accumulators and epilogue: warp w reads TMEM lanes 32 (w % 4) ..
    const int quarter = warp & 3;
    const int r = m0 + quarter * 32 + lane;
    int et[4] = {0, 0, 0, 0}, eref = -100000;
    for (int t = 0; t < row.nterms; ++t) {
      et[t] = r < nt ? aexp[row.t[t].a_row0 + r] : 0;
      eref = max(eref, et[t]);
    }
    float hi[kOzBN], lo[kOzBN];
#pragma unroll
    for (int c = 0; c < kOzBN; ++c) hi[c] = lo[c] = 0.f;
    bool ok = true;
    for (int seg = 0; seg < nseg && ok; ++seg) {
      ok = tc_mb_wait(&seg_full, seg & 1, status) && !*(volatile int*)&abort_flag;
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) { atomicExch(&abort_flag, 1); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int t = seg / segs_per_term;
#pragma unroll 1
      for (int l = 0; l < kOzLevels; ++l) {
        const float w = oz_pow2(et[t] - eref - kOzW * (l + 2));
#pragma unroll
        for (int cc = 0; cc < kOzBN / 16; ++cc) {
          uint32_t v[16];
          const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(l * 64 + cc * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(ta));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) oz_acc(hi[cc * 16 + q], lo[cc * 16 + q], __fmul_rn(__uint_as_float(v[q]), w));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_saddr(&seg_free)) : "memory");
    }
    // ---- epilogue: y = alpha (2^(eref + f_s) (hi + lo) + identity terms) + beta aux
    if (ok && r < nt) {
      const size_t vs = (size_t)T4 * nt;
#pragma unroll
      for (int c = 0; c < kOzBN; ++c) {  // unrolled: hi / lo stay in registers
        const int col = n0 + c;
        if (col >= 2 * S) continue;
        const int s = col < S ? col : col - S;
        const bool im = col >= S;
        double val = ldexp((double)hi[c] + (double)lo[c], eref + fexp[s]);
        const cd* xs = x + (size_t)s * vs;
        const cd* as = aux ? aux + (size_t)s * vs : nullptr;
        for (int e = 0; e < row.nid; ++e) {
          const cd* src = row.id_src[e] == 0 ? xs : as;
          const cd q = src[(size_t)row.id_trace[e] * nt + r];
          val += row.id_sign[e] * (im ? q.y : q.x);
        }
        val *= alpha;
        if (beta != 0.0) {
          const cd q = as[(size_t)row.out * nt + r];
          val += beta * (im ? q.y : q.x);
        }
        reinterpret_cast<double*>(y + (size_t)s * vs + (size_t)row.out * nt + r)[im ? 1 : 0] = val;
      }
    }
  }
  __syncthreads();
  // teardown: every MMA has completed (done), every issued copy has landed, then TMEM is freed
  if (threadIdx.x == 32) tc_mb_wait(&done, 0, status);
  if (threadIdx.x == 0)
    for (int it = consumed; it < issued; ++it) tc_mb_wait(&full[it % kOzStages], (it / kOzStages) & 1, status);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---- host side -----------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool get_encode() {
  if (g_encode) return true;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn) return false;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

// 2D FP16 tensor map: rows x cols (ld halves per row, ld * 2 a multiple of 16), box kTcBK x box_rows
bool tc_make_map(CUtensorMap* m, const void* base, size_t rows, int cols, int ld, int box_rows) {
  if (!get_encode()) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_ld(int nt) { return (2 * nt + 63) / 64 * 64; }

cudaError_t launch_tc_blocks(const cd* blocks, size_t nrows, int nt, int ld, double scale, __half* hi, __half* lo,
                             cudaStream_t s) {
  tc_blocks_kernel<<<2432, 256, 0, s>>>(blocks, nrows, nt, ld, scale, hi, lo);
  return cudaGetLastError();
}
cudaError_t launch_max_abs(const cd* v, size_t n, unsigned long long* out, cudaStream_t s) {
  max_abs_kernel<<<1216, 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}
cudaError_t launch_tc_scale(const cd* x, size_t per_src, int nsrc, int eA, float* scale, float* inv, cudaStream_t s) {
  tc_source_scale_kernel<<<nsrc, 256, 0, s>>>(x, per_src, eA, scale, inv);
  return cudaGetLastError();
}
cudaError_t launch_tc_stage(const TcKey* keys, int nkeys, const cd* x, int nt, int T4, int S, int ld,
                            const float* scale, __half* hi, __half* lo, cudaStream_t s) {
  tc_stage_kernel<<<2432, 256, 0, s>>>(keys, nkeys, x, nt, T4, S, ld, scale, hi, lo);
  return cudaGetLastError();
}

size_t tc_smem_bytes(int bn) { return (size_t)kTcStages * (kTcBM * kTcBK * 2 + bn * kTcBK * 2) + 1024; }

cudaError_t launch_tc_apply(int bn, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
                            const CUtensorMap& blo, const TcRow* rows, int nrows, int nt, int T4, int S, int npass,
                            const float* inv, const cd* x, const cd* aux, cd* y, double alpha, double beta,
                            int* status, cudaStream_t s) {
  const int mt = (nt + kTcBM - 1) / kTcBM;
  const int nn = (2 * S + bn - 1) / bn;
  dim3 grid(mt, nn, nrows);
  const size_t smem = tc_smem_bytes(bn);
  cudaError_t e;
  if (bn == 64) {
    e = smem_limit_max(reinterpret_cast<const void*>(tc_apply_kernel<64>));
    if (e == cudaSuccess)
      tc_apply_kernel<64><<<grid, 128, smem, s>>>(ahi, alo, bhi, blo, rows, nt, T4, S, npass, inv, x, aux, y, alpha,
                                                 beta, status);
  } else if (bn == 128) {
    e = smem_limit_max(reinterpret_cast<const void*>(tc_apply_kernel<128>));
    if (e == cudaSuccess)
      tc_apply_kernel<128><<<grid, 128, smem, s>>>(ahi, alo, bhi, blo, rows, nt, T4, S, npass, inv, x, aux, y, alpha,
                                                  beta, status);
  } else {
    e = smem_limit_max(reinterpret_cast<const void*>(tc_apply_kernel<256>));
    if (e == cudaSuccess)
      tc_apply_kernel<256><<<grid, 128, smem, s>>>(ahi, alo, bhi, blo, rows, nt, T4, S, npass, inv, x, aux, y, alpha,
                                                  beta, status);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t oz_smem_bytes() { return (size_t)kOzStages * kOzP * (kTcBM * kTcBK * 2 + kOzBN * kTcBK * 2) + 1024; }
int oz_slices() { return kOzP; }
int oz_bn() { return kOzBN; }

cudaError_t launch_oz_blocks(const cd* blocks, size_t nrows, int nt, int ld, __half* out, int* ex, cudaStream_t s) {
  oz_blocks_kernel<<<1216, 256, 0, s>>>(blocks, nrows, nt, ld, out, ex);
  return cudaGetLastError();
}
cudaError_t launch_oz_source_exp(const cd* x, size_t per_src, int nsrc, int* fexp, cudaStream_t s) {
  oz_source_exp_kernel<<<nsrc, 256, 0, s>>>(x, per_src, fexp);
  return cudaGetLastError();
}
cudaError_t launch_oz_stage(const TcKey* keys, int nkeys, const cd* x, int nt, int T4, int S, int ld, const int* fexp,
                            size_t slice_rows, __half* out, cudaStream_t s) {
  oz_stage_kernel<<<2432, 256, 0, s>>>(keys, nkeys, x, nt, T4, S, ld, fexp, slice_rows, out);
  return cudaGetLastError();
}
cudaError_t launch_oz_apply(const CUtensorMap& tmA, const CUtensorMap& tmX, const TcRow* rows, int nrows, int nt, int T4,
                            int S, int a_slice_rows, int x_slice_rows, const int* aexp, const int* fexp, const cd* x,
                            const cd* aux, cd* y, double alpha, double beta, int* status, cudaStream_t s) {
  dim3 grid((nt + kTcBM - 1) / kTcBM, (2 * S + kOzBN - 1) / kOzBN, nrows);
  cudaError_t e = smem_limit_max(reinterpret_cast<const void*>(oz_apply_kernel));
  if (e != cudaSuccess) return e;
  oz_apply_kernel<<<grid, kOzThreads, oz_smem_bytes(), s>>>(tmA, tmX, rows, nt, T4, S, a_slice_rows, x_slice_rows, aexp,
                                                            fexp, x, aux, y, alpha, beta, status);
  return cudaGetLastError();
}

}  // namespace pt
