// Local solves (H^l)^{-1} for a batch of sources (Algorithm 2, "solve local
// problems", and the reconstruction of Section 2.3), in FP32 with the Schur
// inverses of the FP64 block factorization rounded to complex64.
//
//   forward  y_i = Sinv_i (f_i - W_i o y_{i-1}),
//   backward x_i = y_i - Sinv_i (E_i o x_{i+1}),      i = 0 .. n_t - 1.
//
// With many sources the chain of 2 n_t - 1 dependent steps becomes, per
// step, one dense nloc x nloc by nloc x GW complex product: one CTA owns one
// (layer, group of GW sources) pair, stages Sinv_i in shared memory once per
// step (cp.async, double-buffered while it fits) and applies it to all GW
// sources, so the factor is read once per group instead of once per source.
// Thread layout: lane = (row sub-group, source); a thread keeps its rows'
// chain state in registers, so the only shared data are Sinv_i and the
// step's right-hand sides V (one barrier after V is written, one after the
// product).
#include <algorithm>
#include <type_traits>

#include "pt_common.cuh"

namespace pt {

constexpr int kBatchThreads = 512;  // 16 warps
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr size_t kBatchSmemMax = 227 * 1024;
constexpr int kLdr = 120;  // shared-memory row pitch of Sinv (>= kMaxNloc, even): row offsets are constants
static_assert(kLdr >= kMaxNloc && kLdr % 2 == 0, "Sinv row pitch");

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Rows of the local problem with a role in the interface coupling (at most
// two of them belong to one thread): MODE 0 emits -x there into a trace of
// P b; MODE 1 adds the forcing sign/h^2 (u_down + u_up) of a trace.
struct BatchSlot {
  int a;        // register slot (row r0 + a * RSTEP), -1 if unused
  int trace;    // MODE 0: output trace index in [0, 2T); MODE 1: forcing trace in [0, T)
  double sign;  // MODE 1 forcing sign (+-1/h^2)
};

template <int MODE, int GW, int RW>
__global__ void __launch_bounds__(kBatchThreads, 1)
    layer_solve_batch_kernel(Geometry g, const LayerInfo* __restrict__ layers, const cf* __restrict__ Shi,
                             const cf* __restrict__ Whi, const cf* __restrict__ Ehi, const cd* __restrict__ f,
                             const cd* __restrict__ xtr, cf* __restrict__ Yst, size_t ylayer, cd* __restrict__ out,
                             const int* __restrict__ nzflag, int nsrc, int nmax, int dbuf) {
  constexpr int RG = 32 / GW;        // row sub-groups in a warp
  constexpr int RSTEP = kBatchWarps * RG;  // distance between the rows of one thread
  // RW rows per thread: RW * RSTEP >= nloc of every layer (checked by the launcher)
  extern __shared__ __align__(16) unsigned char smem[];
  const int l = blockIdx.x, grp = blockIdx.y;
  const LayerInfo L = layers[l];
  const int n = L.nloc, nt = g.nt, T = 2 * (g.L - 1);
  const size_t T4n = (size_t)2 * T * nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sj = lane % GW, rq = lane / GW;
  const int s = grp * GW + sj;
  const bool sval = s < nsrc;
  const bool fnz = sval && nzflag[(size_t)s * g.L + l] != 0;
  const int r0 = warp * RG + rq;
  const int npair = (n + 1) >> 1;
  // [S0][S1 (double buffering)][V][tail]: buffers of nloc_max rows at pitch kLdr; rows past n
  // of a buffer (read by the product loop, results dropped) stay inside the allocation
  cf* S0 = reinterpret_cast<cf*>(smem);
  cf* S1 = dbuf ? S0 + (size_t)nmax * kLdr : S0;
  float4* V = reinterpret_cast<float4*>(S1 + (size_t)nmax * kLdr);  // [npair][GW]: (v_2p, v_2p+1)
  float2* V2 = reinterpret_cast<float2*>(V);

  if (MODE == 0 && !__syncthreads_or(fnz)) {
    // f^l = 0 for every source of the group: its local potentials vanish
    for (int q = threadIdx.x; q < GW * nt; q += kBatchThreads) {
      const int ss = grp * GW + q / nt, k = q % nt;
      if (ss >= nsrc) continue;
      cd* b = out + (size_t)ss * T4n;
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

  // the padding column (odd n) of both Sinv buffers and the padding row of V stay zero
  if (n & 1) {
    for (int r = threadIdx.x; r < n; r += kBatchThreads) {
      S0[(size_t)r * kLdr + n] = make_float2(0.f, 0.f);
      S1[(size_t)r * kLdr + n] = make_float2(0.f, 0.f);
    }
    for (int j = threadIdx.x; j < GW; j += kBatchThreads) V2[((size_t)(npair - 1) * GW + j) * 2 + 1] = make_float2(0.f, 0.f);
  }

  // roles of this thread's rows
  BatchSlot slot[2] = {{-1, 0, 0.0}, {-1, 0, 0.0}};
  {
    const double ih2 = 1.0 / (g.h * g.h);
    auto add = [&](int row, int trace, double sign) {
      if (row < r0 || (row - r0) % RSTEP != 0) return;
      const BatchSlot v{(row - r0) / RSTEP, trace, sign};
      if (slot[0].a < 0) slot[0] = v;
      else slot[1] = v;
    };
    if (MODE == 0) {
      if (L.has_bot) { add(L.row[2], 2 * l, 0.0); add(L.row[3], 2 * l + 1, 0.0); }
      if (L.has_top) { add(L.row[0], T + 2 * (l - 1), 0.0); add(L.row[1], T + 2 * (l - 1) + 1, 0.0); }
    } else {
      if (L.has_top) { add(L.row[1], 2 * (l - 1), ih2); add(L.row[0], 2 * (l - 1) + 1, -ih2); }
      if (L.has_bot) { add(L.row[3], 2 * l, -ih2); add(L.row[2], 2 * l + 1, ih2); }
    }
  }

  const cd* fs = f + (size_t)(sval ? s : 0) * g.Nz * nt;
  const cd* xs = MODE == 1 ? xtr + (size_t)(sval ? s : 0) * T4n : nullptr;
  cf* Yg = Yst + (size_t)(l * gridDim.y + grp) * ylayer;
  const int nsteps = 2 * nt - 1;
  auto col = [&](int st) { return st < nt ? st : nt - 2 - (st - nt); };

  auto stage = [&](int st, cf* dst) {
    const cf* src = Shi + L.sinv_off + (size_t)col(st) * n * n;
    for (int r = warp; r < n; r += kBatchWarps)
      for (int k = lane; k < n; k += 32) cp_async8(dst + r * kLdr + k, src + (size_t)r * n + k);
    cp_async_commit();
  };

  cf yv[RW];    // chain state of my rows: y_{i-1} (forward) / x_{i+1} (backward)
  cf cw[RW];    // W_i or E_i of my rows (prefetched)
  cd fv[RW];    // f_i of my rows (prefetched, forward)
  cf ys[RW];    // stored y_i of my rows (prefetched, backward)
  cd tv[2][2];  // forcing traces (down, up) of my slots (MODE 1, prefetched)
#pragma unroll
  for (int a = 0; a < RW; ++a) {
    yv[a] = make_float2(0.f, 0.f);
    cw[a] = make_float2(0.f, 0.f);
    fv[a] = make_double2(0, 0);
    ys[a] = make_float2(0.f, 0.f);
  }
  tv[0][0] = tv[0][1] = tv[1][0] = tv[1][1] = make_double2(0, 0);

  // stored forward iterates of a backward step; issued after the previous step has consumed ys
  auto prefetch_y = [&](int st) {
    const int i = col(st);
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      const int r = r0 + RSTEP * a;
      if (r < n) ys[a] = Yg[((size_t)i * n + r) * GW + sj];
    }
  };
  auto prefetch = [&](int st) {
    const int i = col(st);
    const bool fwd = st < nt;
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      const int r = r0 + RSTEP * a;
      if (r < n) {
        cw[a] = __ldg((fwd ? Whi : Ehi) + L.coef_off + (size_t)i * n + r);
        if (fwd) {
          cd v = make_double2(0, 0);
          if (fnz && r >= L.pad_top && r < L.pad_top + L.n) v = fs[(size_t)(L.start + r - L.pad_top) * nt + i];
          fv[a] = v;
        }
      }
    }
    if (MODE == 1 && fwd && sval) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (slot[q].a >= 0) {
          tv[q][0] = xs[(size_t)slot[q].trace * nt + i];
          tv[q][1] = xs[(size_t)(T + slot[q].trace) * nt + i];
        }
    }
  };

  // one step of the chain; FWD is a compile-time flag so that the source values
  // (forward only) and the stored iterates (backward only) never hold registers together
  auto step = [&](auto fwd_tag, int st) {
    constexpr bool fwd = decltype(fwd_tag)::value;
    const int i = col(st);
    cf* Sc = (dbuf && (st & 1)) ? S1 : S0;
    // (a) right-hand sides of this step for my rows
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      const int r = r0 + RSTEP * a;
      if (r < n) {
        float vr, vi;
        if constexpr (fwd) {
          cd fd = fv[a];
          if (MODE == 1) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
              if (slot[q].a == a) fd = cadd(fd, cscale(cadd(tv[q][0], tv[q][1]), slot[q].sign));
          }
          vr = (float)fd.x;
          vi = (float)fd.y;
          if (i > 0) {
            vr -= cw[a].x * yv[a].x - cw[a].y * yv[a].y;
            vi -= cw[a].x * yv[a].y + cw[a].y * yv[a].x;
          }
        } else {
          vr = cw[a].x * yv[a].x - cw[a].y * yv[a].y;
          vi = cw[a].x * yv[a].y + cw[a].y * yv[a].x;
        }
        V2[((size_t)(r >> 1) * GW + sj) * 2 + (r & 1)] = make_float2(vr, vi);
      }
    }
    if (st + 1 < nsteps) prefetch(st + 1);
    cp_async_wait_all();
    __syncthreads();
    if (dbuf && st + 1 < nsteps) stage(st + 1, (st & 1) ? S0 : S1);
    // (b) acc = Sinv_i V for my rows and my source.  Row a of this thread sits at a
    // constant offset a * RSTEP * kLdr from its first row; rows past n read padding
    // inside the allocation (results dropped), so the loop has no predicates.
    float ar[RW], ai[RW];
#pragma unroll
    for (int a = 0; a < RW; ++a) { ar[a] = 0.f; ai[a] = 0.f; }
    {
      const float4* sr = reinterpret_cast<const float4*>(Sc + r0 * kLdr);
      const float4* vp = V + sj;
#pragma unroll 1
      for (int p = 0; p < npair; ++p) {
        const float4 v = vp[p * GW];
#pragma unroll
        for (int a = 0; a < RW; ++a) {
          const float4 sp = sr[a * (RSTEP * kLdr / 2) + p];
          ar[a] = fmaf(sp.x, v.x, ar[a]);
          ai[a] = fmaf(sp.x, v.y, ai[a]);
          ar[a] = fmaf(-sp.y, v.y, ar[a]);
          ai[a] = fmaf(sp.y, v.x, ai[a]);
          ar[a] = fmaf(sp.z, v.z, ar[a]);
          ai[a] = fmaf(sp.z, v.w, ai[a]);
          ar[a] = fmaf(-sp.w, v.w, ar[a]);
          ai[a] = fmaf(sp.w, v.z, ai[a]);
        }
      }
    }
    // (c) the step's result for my rows
#pragma unroll
    for (int a = 0; a < RW; ++a) {
      const int r = r0 + RSTEP * a;
      if (r < n) {
        if constexpr (fwd) {
          yv[a] = make_float2(ar[a], ai[a]);
          Yg[((size_t)i * n + r) * GW + sj] = yv[a];
        } else {
          yv[a] = make_float2(ys[a].x - ar[a], ys[a].y - ai[a]);
        }
      }
    }
    if (sval && (!fwd || i == nt - 1)) {
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int a = 0; a < RW; ++a)
            if (slot[q].a == a)
              out[(size_t)s * T4n + (size_t)slot[q].trace * nt + i] = make_double2(-(double)yv[a].x, -(double)yv[a].y);
      } else {
#pragma unroll
        for (int a = 0; a < RW; ++a) {
          const int r = r0 + RSTEP * a;
          if (r < n && r >= L.pad_top && r < L.pad_top + L.n)
            out[(size_t)s * g.Nz * nt + (size_t)(L.start + r - L.pad_top) * nt + i] =
                make_double2((double)yv[a].x, (double)yv[a].y);
        }
      }
    }
    if (st + 1 < nsteps && st + 1 >= nt) prefetch_y(st + 1);
    __syncthreads();
    if (!dbuf && st + 1 < nsteps) stage(st + 1, S0);
  };

  stage(0, S0);
  prefetch(0);
  for (int st = 0; st < nt; ++st) step(std::true_type{}, st);
  for (int st = nt; st < nsteps; ++st) step(std::false_type{}, st);
}

// Group width for a launch: wide groups (fewer Sinv reads per source) while
// the grid still covers the GPU, narrow ones when few (layer, group) pairs exist.
static int batch_group_width(int mode, int L, int nsrc) {
  if (mode == 0) return 8;  // point sources usually excite one layer only
  const int sms = 152;
  if ((long)L * ((nsrc + 31) / 32) >= sms * 3 / 4) return 32;
  if ((long)L * ((nsrc + 15) / 16) >= sms * 3 / 4) return 16;
  return 8;
}

// Shared memory of one CTA: Sinv buffers (nloc_max rows at pitch kLdr), V, and a
// tail so that the rows_read = RW * RSTEP rows read from the last buffer stay inside.
static size_t batch_smem_bytes(int nloc_max, int gw, int rows_read, int* dbuf) {
  const size_t buf = (size_t)nloc_max * kLdr * sizeof(cf);
  const size_t v = (size_t)((nloc_max + 1) / 2) * gw * sizeof(float4);
  auto total = [&](int nbuf) {
    return std::max<size_t>(nbuf * buf + v, (nbuf - 1) * buf + (size_t)rows_read * kLdr * sizeof(cf));
  };
  const bool two = total(2) <= kBatchSmemMax;
  if (dbuf) *dbuf = two ? 1 : 0;
  return total(two ? 2 : 1);
}

template <int MODE, int GW, int RW>
static cudaError_t go_batch(const Geometry& g, const LayerInfo* layers, int nloc_max, const cf* Shi, const cf* Whi,
                            const cf* Ehi, const cd* f, const cd* xtr, cf* Y, cd* out, const int* flag, int nsrc,
                            cudaStream_t s) {
  int dbuf = 0;
  const size_t smem = batch_smem_bytes(nloc_max, GW, RW * kBatchWarps * (32 / GW), &dbuf);
  if (smem > kBatchSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = smem_limit_max(reinterpret_cast<const void*>(layer_solve_batch_kernel<MODE, GW, RW>));
  if (e != cudaSuccess) return e;
  const size_t ylayer = (size_t)g.nt * nloc_max * GW;
  dim3 grid(g.L, (nsrc + GW - 1) / GW);
  layer_solve_batch_kernel<MODE, GW, RW><<<grid, kBatchThreads, smem, s>>>(g, layers, Shi, Whi, Ehi, f, xtr, Y,
                                                                           ylayer, out, flag, nsrc, nloc_max, dbuf);
  return cudaGetLastError();
}

// rows per thread: the smallest RW with RW * RSTEP >= nloc_max
template <int MODE, int GW>
static cudaError_t go_rows(const Geometry& g, const LayerInfo* layers, int nloc_max, const cf* Shi, const cf* Whi,
                           const cf* Ehi, const cd* f, const cd* xtr, cf* Y, cd* out, const int* flag, int nsrc,
                           cudaStream_t s) {
  constexpr int RSTEP = kBatchWarps * (32 / GW);
  const int rw = (nloc_max + RSTEP - 1) / RSTEP;
#define PT_GO(R)                                                                                          \
  if (rw == R) return go_batch<MODE, GW, R>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Y, out, flag, nsrc, s);
  if constexpr (GW == 32) {
    PT_GO(1) PT_GO(2) PT_GO(3) PT_GO(4) PT_GO(5) PT_GO(6) PT_GO(7) PT_GO(8)
  } else if constexpr (GW == 16) {
    PT_GO(1) PT_GO(2) PT_GO(3) PT_GO(4)
  } else {
    PT_GO(1) PT_GO(2)
  }
#undef PT_GO
  return cudaErrorInvalidValue;
}

// gw_opt: 0 = automatic, else 8, 16 or 32 sources per CTA.  The Y scratch
// holds round_up(nsrc, 32) sources' iterates in complex64.
cudaError_t launch_layer_solve_batch(int mode, const Geometry& g, const LayerInfo* layers, int nloc_max,
                                     const cf* Shi, const cf* Whi, const cf* Ehi, const cd* f, const cd* xtr, cd* Y,
                                     cd* out, const int* flag, int nsrc, int gw_opt, cudaStream_t s) {
  static_assert(kMaxNloc <= 8 * kBatchWarps, "row slots per thread");
  if (nloc_max > kMaxNloc || nloc_max < 1) return cudaErrorInvalidValue;
  cf* Yc = reinterpret_cast<cf*>(Y);
  const int gw = gw_opt ? gw_opt : batch_group_width(mode, g.L, nsrc);
  if (mode == 0) {
    if (gw == 32) return go_rows<0, 32>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Yc, out, flag, nsrc, s);
    if (gw == 16) return go_rows<0, 16>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Yc, out, flag, nsrc, s);
    return go_rows<0, 8>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Yc, out, flag, nsrc, s);
  }
  if (gw == 32) return go_rows<1, 32>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Yc, out, flag, nsrc, s);
  if (gw == 16) return go_rows<1, 16>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Yc, out, flag, nsrc, s);
  return go_rows<1, 8>(g, layers, nloc_max, Shi, Whi, Ehi, f, xtr, Yc, out, flag, nsrc, s);
}

}  // namespace pt
