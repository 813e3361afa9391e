// Host side of the C ABI declared in include/polartrace.h.
//
// pt_create runs Algorithm 1 (offline) and builds the operator tables of the
// permuted polarized jump system P M = D + R (Section 3.5); pt_solve runs
// Algorithm 2 with flexible GMRES (right preconditioned by Algorithm 4,
// Section 4.2) driven from the host, one stream synchronisation per iteration.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/polartrace.h"
#include "pt_common.cuh"

namespace pt {
cudaError_t launch_check_medium(const double*, size_t, int*, cudaStream_t);
cudaError_t launch_coef(const Geometry&, const LayerInfo*, const double*, cd*, cd*, cudaStream_t);
cudaError_t launch_factor(const Geometry&, const LayerInfo*, int, const double*, cd*, int*, cudaStream_t);
cudaError_t launch_extract(const Geometry&, const LayerInfo*, const ExtractTask*, int, int, int, const cd*,
                           const cd*, const cd*, cd*, size_t, cd*, cudaStream_t);
cudaError_t launch_apply_mode(int, int, int, int, const ApplyRow*, int, const void*, const void*, const cd*,
                              const cd*, cd*, int, int, double, double, cudaStream_t);
cudaError_t launch_split_blocks(const cd*, int, int, size_t, cf*, cf*, cudaStream_t);
cudaError_t launch_split_sinv(const cd*, size_t, cf*, cf*, cudaStream_t);
cudaError_t launch_layer_nonzero(const Geometry&, const LayerInfo*, const cd*, int*, int*, int, cudaStream_t);
cudaError_t launch_layer_solve(int, const Geometry&, const LayerInfo*, const cd*, const cd*, const cd*, const cd*,
                               const cd*, cd*, size_t, cd*, const int*, int, cudaStream_t);
cudaError_t launch_layer_solve2(int, bool, const Geometry&, const LayerInfo*, const cd*, const cf*, const cf*,
                                const cd*, const cd*, const cd*, const cd*, cd*, size_t, cd*, const int*, int,
                                cudaStream_t);
cudaError_t launch_layer_solve_df(int, const Geometry&, const LayerInfo*, const cf*, const cf*, const cf*, const cf*,
                                  const cf*, const cf*, const cd*, const cd*, cd*, size_t, cd*, const int*, int,
                                  cudaStream_t);
int dot_chunks(size_t N);
size_t plr_scratch_per_cta(int nt);
int plr_max_k();
cudaError_t launch_plr_compress(int, const cd*, const int*, int, int, double, int, cd*, int, PlrLeaf*, int, int*, cd*,
                                int*, cudaStream_t);
cudaError_t launch_plr_apply(bool, int, int, int, const ApplyRow*, int, const void*, const void*, const PlrLeaf*,
                             const PlrTask*, int, const int*, const int*, const int*, const int*, cd*, int, const cd*,
                             const cd*, cd*, int, double, double, cudaStream_t);
cudaError_t launch_pool_to_fp32(const cd*, cf*, size_t, cudaStream_t);
bool tc_make_map(CUtensorMap*, const void*, size_t, int, int, int);
int tc_ld(int nt);
cudaError_t launch_tc_blocks(const cd*, size_t, int, int, double, __half*, __half*, cudaStream_t);
cudaError_t launch_max_abs(const cd*, size_t, unsigned long long*, cudaStream_t);
cudaError_t launch_tc_scale(const cd*, size_t, int, int, float*, float*, cudaStream_t);
cudaError_t launch_tc_stage(const TcKey*, int, const cd*, int, int, int, int, const float*, __half*, __half*,
                            cudaStream_t);
cudaError_t launch_tc_apply(int, const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const CUtensorMap&,
                            const TcRow*, int, int, int, int, int, const float*, const cd*, const cd*, cd*, double,
                            double, int*, cudaStream_t);
cudaError_t launch_layer_solve_f32(int, const Geometry&, const LayerInfo*, int, const cf*, const cf*, const cf*,
                                   const cd*, const cd*, cd*, size_t, cd*, const int*, const int*, int, int*, int,
                                   cudaStream_t);
cudaError_t launch_layer_solve_batch(int, const Geometry&, const LayerInfo*, int, const cf*, const cf*, const cf*,
                                     const cd*, const cd*, cd*, cd*, const int*, int, int, cudaStream_t);
cudaError_t nn_forward(const __nv_bfloat16*, const float*, const float*, long, int, float*, float*, float*,
                       cudaStream_t);
cudaError_t nn_backward(const __nv_bfloat16*, const float*, long, int, const float*, const float*, const float*,
                        const float*, float*, float*, float*, float*, double*, cudaStream_t);
cudaError_t nn_to_bf16(const float*, __nv_bfloat16*, cudaStream_t);
cudaError_t nn_adam(float*, float*, float*, const float*, __nv_bfloat16*, double, int, cudaStream_t);
cudaError_t nn_rms(const cd*, int, size_t, double*, cudaStream_t);
cudaError_t nn_features(const cd*, int, int, int, int, const double*, float*, long, cudaStream_t);
cudaError_t nn_unfeatures(const float*, int, int, int, int, const double*, cd*, bool, cudaStream_t);
cudaError_t nn_gather(const float*, long, const int*, int, int, int, float*, cudaStream_t);
cudaError_t nn_sub(const cd*, const cd*, cd*, size_t, cudaStream_t);
cudaError_t nn_sumsq(const float*, long, double*, cudaStream_t);
cudaError_t nn_scale(float*, long, float, cudaStream_t);
bool launch_apply_f32_rows(int, int, int, const ApplyRow*, int, const void*, const cd*, const cd*, cd*, int, double,
                           double, cudaStream_t, cudaError_t*);
size_t chunk_work_bytes(int, int, int);
cudaError_t launch_chunk_transfer(const Geometry&, const LayerInfo*, const cd*, const cd*, const cd*, int, int, cd*,
                                  cf*, cudaStream_t);
cudaError_t launch_to_c64(const cd*, size_t, cf*, cudaStream_t);
cudaError_t launch_layer_solve_chunked(int, const Geometry&, const LayerInfo*, int, int, const cf*, const cf*,
                                       const cf*, const cf*, const cf*, const cd*, cf*, cd*, size_t, cd*, cf*,
                                       const int*, cf*, int, int*, cudaStream_t);
cudaError_t launch_prep_inputs(const cd*, int, int, int, bool, void*, cudaStream_t);
cudaError_t launch_apply_lowp(int, int, int, int, const ApplyRow*, int, const void*, const void*, const void*,
                              const cd*, const cd*, cd*, int, int, double, double, cudaStream_t);
cudaError_t launch_blocks_h16(const cd*, int, int, size_t, __half2*, float*, cudaStream_t);
bool launch_sweep_f32(int, int, int, int, const ApplyRow*, const void*, const float*, const cd*, cd*, cf*, int,
                      unsigned*, int*, cudaStream_t, cudaError_t*);
cudaError_t launch_volume_residual(const Geometry&, const double*, const cd*, const cd*, int, double*, cudaStream_t);
cudaError_t launch_dots(const cd*, int, size_t, const cd*, int, cd*, cd*, int, cd*, int, int, int, cudaStream_t);
cudaError_t launch_update(const cd*, int, size_t, cd*, int, const cd*, int, cudaStream_t);
cudaError_t launch_norm_scale(const cd*, size_t, int, double*, cd*, int, int, int, int, cd*, size_t, double*,
                              cudaStream_t);
cudaError_t launch_givens(int, int, int, cd*, double*, cd*, cd*, double*, cudaStream_t);
cudaError_t launch_lsq_combine(int, int, const int*, const cd*, const cd*, cd*, const cd*, size_t, cd*,
                               cudaStream_t);
cudaError_t launch_sub(const cd*, const cd*, cd*, size_t, cudaStream_t);
int oz_slices();
int oz_bn();
cudaError_t launch_oz_blocks(const cd*, size_t, int, int, __half*, int*, cudaStream_t);
cudaError_t launch_oz_source_exp(const cd*, size_t, int, int*, cudaStream_t);
cudaError_t launch_oz_stage(const TcKey*, int, const cd*, int, int, int, int, const int*, size_t, __half*,
                            cudaStream_t);
cudaError_t launch_oz_apply(const CUtensorMap&, const CUtensorMap&, const TcRow*, int, int, int, int, int, int,
                            const int*, const int*, const cd*, const cd*, cd*, double, double, int*, cudaStream_t);
}  // namespace pt

using namespace pt;

static thread_local std::string g_last_error;
// set on the worker threads of pt_solve_many: contexts that share the GPU take no cooperative launches
static thread_local bool g_shared_gpu = false;

static pt_status fail(pt_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define PT_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(PT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

constexpr size_t kAlign = 256;
constexpr int kExtractSlots = 152;
constexpr int kApplyRowsSweep = 8;   // rows per CTA for the sweep steps
constexpr int kApplyRowsWide = 16;   // rows per CTA for R and the matvec
constexpr double kRelax = 1e4;       // FP32 GMRES matvecs once ||r|| <= kRelax tol ||b|| (mixed FP32 form)
constexpr int kPlrCap = 512;         // leaves per compressed block
constexpr int kPlrSlots = 152;       // CTAs of the compression kernel

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Plan {
  Geometry g{};
  int L = 0, nt = 0, Nz = 0, T = 0, T4 = 0;
  int ld32 = 0;  // row stride of the FP32 block copies (n_t rounded up to 4: 16-byte aligned rows)
  size_t N = 0;  // entries of one polarized-trace vector
  int nloc_max = 0;
  std::vector<LayerInfo> layers;
  std::vector<ExtractTask> tasks;
  size_t sinv_elems = 0, coef_elems = 0;
  // partitioned low-rank blocks
  bool plr = false;
  int rmax = 0, oversample = 0, ntiles = 0;
  std::vector<int> plr_blocks;  // absolute block slots (layer * 16 + jk) that exist
  size_t plr_task_cap = 0;      // projection tasks of one operator table, upper bound
  // tensor-core form
  bool tc = false;
  int ldtc = 0;                 // halves per row of the FP16 [Br Bi] rows
  std::vector<TcRow> tc_mv, tc_R, tc_sw;
  std::vector<TcKey> tk_mv, tk_R, tk_sw;
  std::vector<int> tk_sw_off, tk_sw_cnt;
  int tc_keys_max = 0;
  // learned correction: inference buffers for nn_cs sources at a time
  bool learned = false;
  int nn_cs = 0;
  // chunked local solves of the mixed FP32 form: chunks per layer of the right-hand side
  // (one active layer per point source: short chains) and of the reconstruction (every
  // layer at once: about one chunk per SM)
  int kr = 0, kv = 0;
};

pt_status make_plan(const pt_params* p, Plan& P) {
  if (!p) return fail(PT_ERR_ARG, "params is NULL");
  if (p->nx < 1 || p->nz < 1 || p->npml < 1 || p->L < 2 || p->L > kMaxLayers)
    return fail(PT_ERR_ARG, "need nx, nz, npml >= 1 and 2 <= L <= 256");
  if (!(p->h > 0) || !(p->omega > 0) || !(p->pml_C >= 0) || !std::isfinite(p->h) || !std::isfinite(p->omega) ||
      !std::isfinite(p->pml_C))
    return fail(PT_ERR_ARG, "h and omega must be positive, pml_C non-negative, all finite");
  if (p->precision != PT_FP64 && p->precision != PT_MIXED_FP32 && p->precision != PT_MIXED_TC)
    return fail(PT_ERR_ARG, "unknown precision");
  if (p->precision == PT_MIXED_TC && p->plr) return fail(PT_ERR_ARG, "PT_MIXED_TC applies dense blocks (plr = 0)");
  if (p->gs_iters < 1 || p->gs_iters > 16) return fail(PT_ERR_ARG, "gs_iters must be in 1..16");
  if (p->learned != 0 && p->learned != 1) return fail(PT_ERR_ARG, "learned must be 0 or 1");
  if (p->max_sources < 1 || p->max_krylov < 1 || p->max_krylov > 512)
    return fail(PT_ERR_ARG, "max_sources >= 1 and 1 <= max_krylov <= 512");
  P.learned = p->learned == 1;
  P.nt = p->nx + 2 * p->npml;
  P.Nz = p->nz + 2 * p->npml;
  P.L = p->L;
  P.T = 2 * (P.L - 1);
  P.T4 = 4 * (P.L - 1);
  P.N = (size_t)P.T4 * P.nt;
  if (P.learned) {  // inference in chunks of about 64 Ki positions (at least one source)
    const long per = (long)(P.L - 1) * P.nt;
    P.nn_cs = (int)std::max<long>(1, std::min<long>(p->max_sources, 65536 / per));
  }
  P.ld32 = (P.nt + 3) & ~3;
  P.g = Geometry{P.nt, P.Nz, p->npml, P.L, p->h, p->omega, p->pml_C};
  // the caller's rows per layer, or the near-equal split: the first (N_z mod L) layers get one
  // extra row
  const int base = P.Nz / P.L, extra = P.Nz % P.L;
  if (p->layer_rows) {
    long long sum = 0;
    for (int l = 0; l < P.L; ++l) sum += p->layer_rows[l];
    if (sum != P.Nz) return fail(PT_ERR_ARG, "layer_rows must sum to N_z = nz + 2 npml");
  }
  int start = 0;
  P.layers.resize(P.L);
  for (int l = 0; l < P.L; ++l) {
    LayerInfo& I = P.layers[l];
    I.start = start;
    I.n = p->layer_rows ? p->layer_rows[l] : base + (l < extra ? 1 : 0);
    start += I.n;
    I.has_top = l > 0;
    I.has_bot = l < P.L - 1;
    I.pad_top = I.has_top ? p->npml : 0;
    I.pad_bot = I.has_bot ? p->npml : 0;
    I.nloc = I.pad_top + I.n + I.pad_bot;
    I.row[0] = I.has_top ? I.pad_top - 1 : -1;
    I.row[1] = I.has_top ? I.pad_top : -1;
    I.row[2] = I.has_bot ? I.pad_top + I.n - 1 : -1;
    I.row[3] = I.has_bot ? I.pad_top + I.n : -1;
    if (I.n < 3) return fail(PT_ERR_ARG, "every layer needs at least 3 rows");
    if (l > 0 && !(I.start >= p->npml + 1 && I.start <= P.Nz - p->npml - 1))
      return fail(PT_ERR_ARG, "an interface lies in or next to the PML; use fewer or other layers");
    P.nloc_max = std::max(P.nloc_max, I.nloc);
    I.sinv_off = (long long)P.sinv_elems;
    I.coef_off = (long long)P.coef_elems;
    P.sinv_elems += (size_t)P.nt * I.nloc * I.nloc;
    P.coef_elems += (size_t)P.nt * I.nloc;
  }
  if (P.nloc_max > kMaxNloc)
    return fail(PT_ERR_ARG, "a local problem has more than 118 rows (layer rows + 2 n_pml); use more layers");
  if (p->precision == PT_MIXED_FP32) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 152;
    }
    const int kmax = std::max(1, std::min(64, P.nt / 16));  // chunks of at least 16 columns
    P.kr = std::min(kmax, 32);
    P.kv = std::max(1, std::min(kmax, sms / P.L));
  }
  if (p->plr) {
    if (p->plr_rmax < 1 || p->plr_rmax > 31 || !(p->plr_eps > 0) || !std::isfinite(p->plr_eps))
      return fail(PT_ERR_ARG, "plr needs 1 <= plr_rmax <= 31 and plr_eps > 0");
    P.plr = true;
    P.rmax = p->plr_rmax;
    P.oversample = std::min(8, plr_max_k() - 1 - P.rmax);
    P.ntiles = (P.nt + 31) / 32;
    for (int l = 0; l < P.L; ++l) {
      const LayerInfo& I = P.layers[l];
      for (int jj = 0; jj < 4; ++jj)
        for (int kk = 0; kk < 4; ++kk) {
          const bool jo = (jj < 2) ? I.has_top : I.has_bot;
          const bool ko = (kk < 2) ? I.has_top : I.has_bot;
          if (jo && ko) P.plr_blocks.push_back(l * 16 + jj * 4 + kk);
        }
    }
    P.plr_task_cap = (size_t)P.T4 * 4 * kPlrCap;
  }
  // extraction tasks: 32 right-hand sides each
  for (int l = 0; l < P.L; ++l) {
    ExtractTask t{};
    t.layer = l;
    t.nk = 0;
    if (P.layers[l].has_top) { t.kk[t.nk++] = 0; t.kk[t.nk++] = 1; }
    if (P.layers[l].has_bot) { t.kk[t.nk++] = 2; t.kk[t.nk++] = 3; }
    t.w = 32 / t.nk;
    for (int c0 = 0; c0 < P.nt; c0 += t.w) {
      t.c0 = c0;
      P.tasks.push_back(t);
    }
  }
  return PT_OK;
}

struct Persist {
  LayerInfo* layers;
  int* status;
  unsigned* sweep_bar;  // grid-barrier counter of the one-launch sweeps
  cf* sweep_y32;        // complex64 copies of the traces a one-launch sweep writes (mixed FP32 form)
  void* xprep;          // inputs of the FP32 / double-float applies converted once per application
  cf* chunk_T;          // Phi_k, M_k, Psi_k of the chunked local solves: [kr set | kv set][L][K][3][nloc_max^2]
  __half2* blocks_h16;  // mixed FP32 form: FP16 block copies for the preconditioner, rows padded to ld32
  float* bscale;        // and one scale per block row
  cd* W;
  cd* E;
  cd* Sinv;
  cd* blocks;
  cf* blocks_hi;  // mixed form: fl32(B) and fl32(B - hi), rows padded to ld32
  cf* blocks_lo;
  cf* sinv_hi;    // mixed form: double-float split of the local factors
  cf* sinv_lo;
  cf *w_hi, *w_lo, *e_hi, *e_lo;  // mixed form: double-float split of the x-couplings
  ApplyRow* tab_matvec;
  ApplyRow* tab_R;
  ApplyRow* tab_sweep;
  ExtractTask* tasks;
  // PLR
  PlrLeaf* leaves;      // [nblk][kPlrCap]
  int* nleaves;         // [nblk]
  int* plr_ids;         // [nblk] absolute block slots
  cd* pool;             // [nblk][nt * nt] factors
  cf* pool32;           // mixed form: FP32 copy
  int* lr_ord;          // [nblk * cap] ordinal among the low-rank leaves of the block
  int* tile_ptr;        // [L * 16 * ntiles + 1]
  int* tile_leaf;       // CSR entries
  PlrTask* task_mv;     // matvec table
  int* tbase_mv;
  PlrTask* task_R;      // coupling table
  int* tbase_R;
  PlrTask* task_sw;     // sweep steps, (L-1) x 4 rows
  int* tbase_sw;
  // tensor-core form
  __half* tc_ahi;       // [L * 16 * nt][ldtc]
  __half* tc_alo;
  __half* oz_a;         // split products of the restart residual: kOzP slices of [L * 16 * nt][ldtc]
  int* oz_e;            // their row exponents [L * 16 * nt]
  TcRow* tcr_mv;
  TcRow* tcr_R;
  TcRow* tcr_sw;
  TcKey* tck_mv;
  TcKey* tck_R;
  TcKey* tck_sw;
  unsigned long long* tc_max;
  double* m_ext;        // squared slowness on the extended grid (volume residual)
  // learned correction: FP32 master weights, BF16 copy, Adam moments, gradient, loss
  float *nn_theta, *nn_m, *nn_v, *nn_grad;
  __nv_bfloat16* nn_wbf;
  double* nn_loss;
};

Persist carve_persist(const Plan& P, const pt_params* p, void* base, size_t* bytes) {
  Carver c(base);
  Persist q{};
  q.layers = c.take<LayerInfo>(P.L);
  q.status = c.take<int>(64);
  q.sweep_bar = c.take<unsigned>(64);
  q.W = c.take<cd>(P.coef_elems);
  q.E = c.take<cd>(P.coef_elems);
  q.Sinv = c.take<cd>(P.sinv_elems);
  const size_t bel = (size_t)P.L * 16 * P.nt * P.nt;
  q.blocks = c.take<cd>(bel);
  if (p->precision != PT_FP64) {  // FP32 / double-float copies of the blocks for the apply kernels
    const size_t bel32 = (size_t)P.L * 16 * P.nt * P.ld32;
    q.blocks_hi = c.take<cf>(bel32);
    q.blocks_lo = c.take<cf>(bel32);
  }
  if (p->precision != PT_FP64) {  // both mixed forms run the local solves in double-float
    q.sinv_hi = c.take<cf>(P.sinv_elems);
    q.sinv_lo = c.take<cf>(P.sinv_elems);
    q.w_hi = c.take<cf>(P.coef_elems);
    q.w_lo = c.take<cf>(P.coef_elems);
    q.e_hi = c.take<cf>(P.coef_elems);
    q.e_lo = c.take<cf>(P.coef_elems);
  }
  if (p->precision == PT_MIXED_FP32 && !P.plr) {
    q.sweep_y32 = c.take<cf>((size_t)p->max_sources * P.T4 * P.nt);
    q.blocks_h16 = c.take<__half2>((size_t)P.L * 16 * P.nt * P.ld32);
    q.bscale = c.take<float>((size_t)P.L * 16 * P.nt);
  }
  if (p->precision != PT_FP64 && !P.plr) q.xprep = c.take<float4>((size_t)p->max_sources * P.T4 * P.ld32);
  if (P.kr > 0)
    q.chunk_T = c.take<cf>((size_t)P.L * (P.kr + P.kv) * 3 * P.nloc_max * P.nloc_max);
  q.tab_matvec = c.take<ApplyRow>(P.T4);
  q.tab_R = c.take<ApplyRow>(P.T4);
  q.tab_sweep = c.take<ApplyRow>((size_t)(P.L - 1) * 4);
  q.tasks = c.take<ExtractTask>(P.tasks.size());
  if (P.plr) {
    const size_t nb = P.plr_blocks.size();
    q.leaves = c.take<PlrLeaf>(nb * kPlrCap);
    q.nleaves = c.take<int>(nb);
    q.plr_ids = c.take<int>(nb);
    q.pool = c.take<cd>(nb * P.nt * P.nt);
    if (p->precision == PT_MIXED_FP32) q.pool32 = c.take<cf>(nb * P.nt * P.nt);
    q.lr_ord = c.take<int>(nb * kPlrCap);
    q.tile_ptr = c.take<int>((size_t)P.L * 16 * P.ntiles + 1);
    q.tile_leaf = c.take<int>(nb * kPlrCap * (size_t)P.ntiles);
    q.task_mv = c.take<PlrTask>(P.plr_task_cap);
    q.tbase_mv = c.take<int>((size_t)P.T4 * 4);
    q.task_R = c.take<PlrTask>(P.plr_task_cap);
    q.tbase_R = c.take<int>((size_t)P.T4 * 4);
    q.task_sw = c.take<PlrTask>(P.plr_task_cap);
    q.tbase_sw = c.take<int>((size_t)(P.L - 1) * 16);
  }
  if (P.tc) {
    const size_t rowsA = (size_t)P.L * 16 * P.nt;
    q.tc_ahi = c.take<__half>(rowsA * P.ldtc);
    q.tc_alo = c.take<__half>(rowsA * P.ldtc);
    q.tcr_mv = c.take<TcRow>(P.tc_mv.size());
    q.tcr_R = c.take<TcRow>(P.tc_R.size());
    q.tcr_sw = c.take<TcRow>(P.tc_sw.size());
    q.tck_mv = c.take<TcKey>(P.tk_mv.size());
    q.tck_R = c.take<TcKey>(P.tk_R.size());
    q.tck_sw = c.take<TcKey>(P.tk_sw.size());
    q.tc_max = c.take<unsigned long long>(4);
    q.oz_a = c.take<__half>((size_t)oz_slices() * rowsA * P.ldtc);
    q.oz_e = c.take<int>(rowsA);
  }
  q.m_ext = c.take<double>((size_t)P.Nz * P.nt);
  q.nn_theta = c.take<float>(kNnParams);
  q.nn_m = c.take<float>(kNnParams);
  q.nn_v = c.take<float>(kNnParams);
  q.nn_grad = c.take<float>(kNnParams);
  q.nn_wbf = c.take<__nv_bfloat16>(kNnParams);
  q.nn_loss = c.take<double>(4);
  if (bytes) *bytes = c.off;
  return q;
}

size_t setup_slot_elems(const Plan& P) { return (size_t)P.nt * P.nloc_max * 32; }

size_t setup_bytes_of(const Plan& P) {
  Carver c(nullptr);
  int nslots = std::min<int>((int)P.tasks.size(), kExtractSlots);
  c.take<cd>(setup_slot_elems(P) * nslots);
  // the chunk transfer matrices are formed after the extraction, in the same scratch
  return std::max(c.off, chunk_work_bytes(P.L, std::max(P.kr, P.kv), P.nloc_max));
}

// The PLR compressor reuses the setup workspace after the extraction.
size_t plr_setup_bytes(const Plan& P) {
  if (!P.plr) return 0;
  Carver c(nullptr);
  const int nslots = std::min<int>((int)P.plr_blocks.size(), kPlrSlots);
  c.take<cd>(plr_scratch_per_cta(P.nt) * nslots);
  return c.off;
}

struct SolveBufs {
  cd* Y;
  int* nzflag;
  int* nzfirst;  // first grid column of f^l with a non-zero entry
  cf* chunk_bnd; // chunked local solves: y'_b, x''_a, beta, gamma per (source, layer, chunk)
  cf *f32, *tr32, *vol32;  // chunked local solves: complex64 sources, trace forcing and volume
  cd *b, *x, *w, *t, *u1, *V, *Z, *partial, *coef, *H, *sn, *g, *y;
  double *cs, *resid, *nrm;
  int* kk;
  cd *fdev, *udev;  // pt_solve_host staging
  cd* tbuf;         // PLR projections
  __half *tc_bhi, *tc_blo;  // staged tensor-core operands
  float *tc_scale, *tc_inv;
  __half* oz_x;     // staged input slices of the split restart product
  int* oz_f;        // per-source exponents of those inputs
  double* vres;     // volume residual partials
  double* nn_rms;   // learned correction: per-source RMS of the input
  float *nn_X, *nn_A, *nn_Y;  // features, two W x P activation buffers, outputs
};

SolveBufs carve_solve(const Plan& P, int S, int m, bool host_staging, void* base, size_t* bytes) {
  Carver c(base);
  SolveBufs b{};
  const size_t N = P.N;
  // forward iterates of the local solves; the source-batched solves of the tensor-core
  // form keep them in complex64 per (layer, group of up to 32 sources): room for
  // round_up(S, 32) sources in half the bytes
  b.Y = c.take<cd>((size_t)(P.tc ? std::max(S, 16) : S) * P.L * P.nt * P.nloc_max);
  b.nzflag = c.take<int>((size_t)S * P.L);
  b.nzfirst = c.take<int>((size_t)S * P.L);
  if (P.kr > 0) {
    b.chunk_bnd = c.take<cf>((size_t)S * P.L * std::max(P.kr, P.kv) * 4 * P.nloc_max);
    b.f32 = c.take<cf>((size_t)S * P.Nz * P.nt);
    b.tr32 = c.take<cf>((size_t)S * P.N);
    b.vol32 = c.take<cf>((size_t)S * P.Nz * P.nt);
  }
  b.b = c.take<cd>(S * N);
  b.x = c.take<cd>(S * N);
  b.w = c.take<cd>(S * N);
  b.t = c.take<cd>(S * N);
  b.u1 = c.take<cd>(S * N);
  b.V = c.take<cd>((size_t)(m + 1) * S * N);
  b.Z = c.take<cd>((size_t)m * S * N);
  b.partial = c.take<cd>((size_t)S * (m + 1) * dot_chunks(N));
  b.coef = c.take<cd>((size_t)S * (m + 1));
  b.H = c.take<cd>((size_t)S * (m + 1) * m);
  b.sn = c.take<cd>((size_t)S * m);
  b.g = c.take<cd>((size_t)S * (m + 1));
  b.y = c.take<cd>((size_t)S * (m + 1));
  b.cs = c.take<double>((size_t)S * m);
  b.resid = c.take<double>(S);
  b.nrm = c.take<double>(S);
  b.kk = c.take<int>(S);
  b.tbuf = P.plr ? c.take<cd>((size_t)S * P.plr_task_cap * P.rmax) : nullptr;
  if (P.tc) {
    const size_t el = (size_t)P.tc_keys_max * 2 * S * P.ldtc;
    b.tc_bhi = c.take<__half>(el);
    b.tc_blo = c.take<__half>(el);
    b.tc_scale = c.take<float>(S);
    b.tc_inv = c.take<float>(S);
    b.oz_x = c.take<__half>((size_t)oz_slices() * P.tk_mv.size() * 2 * S * P.ldtc);
    b.oz_f = c.take<int>(S);
  }
  b.vres = c.take<double>((size_t)S + (size_t)S * 2 * 512);
  if (P.learned) {
    const size_t Pm = (size_t)P.nn_cs * (P.L - 1) * P.nt;
    b.nn_rms = c.take<double>(S);
    b.nn_X = c.take<float>(kNnCin * Pm);
    b.nn_A = c.take<float>(2 * kNnW * Pm);
    b.nn_Y = c.take<float>(kNnCin * Pm);
  }
  if (host_staging) {
    b.fdev = c.take<cd>((size_t)S * P.Nz * P.nt);
    b.udev = c.take<cd>((size_t)S * P.Nz * P.nt);
  }
  if (bytes) *bytes = c.off;
  return b;
}

// ---- operator tables -------------------------------------------------------
struct TableBuilder {
  const Plan& P;
  int tr(int dir, int iface, int ab) const { return dir * P.T + 2 * iface + ab; }
  static int blk(int l, int jj, int kk) { return l * 16 + jj * 4 + kk; }
  // G_down_j(p) of layer l, p = top pair (interface l-1): B_{j,1} p.A - B_{j,0} p.B
  void down(ApplyRow& r, int l, int jj, int inA, int inB, int inA2 = -1, int inB2 = -1) const {
    r.t[r.nterms++] = ApplyTerm{blk(l, jj, 1), inA, inA2, +1.0};
    r.t[r.nterms++] = ApplyTerm{blk(l, jj, 0), inB, inB2, -1.0};
  }
  // G_up_j(q) of layer l, q = bottom pair (interface l): -B_{j,n+1} q.A + B_{j,n} q.B
  void up(ApplyRow& r, int l, int jj, int inA, int inB, int inA2 = -1, int inB2 = -1) const {
    r.t[r.nterms++] = ApplyTerm{blk(l, jj, 3), inA, inA2, -1.0};
    r.t[r.nterms++] = ApplyTerm{blk(l, jj, 2), inB, inB2, +1.0};
  }
  static void ident(ApplyRow& r, int src, int trace, double sign) {
    r.id_src[r.nid] = src;
    r.id_trace[r.nid] = trace;
    r.id_sign[r.nid] = sign;
    r.nid++;
  }
  static ApplyRow row(int out) {
    ApplyRow r;
    std::memset(&r, 0, sizeof(r));
    r.out = out;
    return r;
  }

  // y = P M x = (D + R) x: the four jump-condition equations of Section 3.5.
  std::vector<ApplyRow> matvec() const {
    std::vector<ApplyRow> v;
    const int L = P.L;
    for (int l = 0; l + 1 < L; ++l) {  // down rows of interface l (layer l): j = n, j = n+1
      for (int jj = 2; jj <= 3; ++jj) {
        ApplyRow r = row(tr(0, l, jj - 2));
        if (l >= 1) down(r, l, jj, tr(1, l - 1, 0), tr(1, l - 1, 1), tr(0, l - 1, 0), tr(0, l - 1, 1));
        up(r, l, jj, tr(1, l, 0), tr(1, l, 1));
        if (jj == 2) { ident(r, 0, tr(1, l, 0), -1.0); ident(r, 0, tr(0, l, 0), -1.0); }
        else ident(r, 0, tr(0, l, 1), -1.0);
        v.push_back(r);
      }
    }
    for (int l = 1; l < L; ++l) {  // up rows of interface l-1 (layer l): j = 0, j = 1
      for (int jj = 0; jj <= 1; ++jj) {
        ApplyRow r = row(tr(1, l - 1, jj));
        down(r, l, jj, tr(0, l - 1, 0), tr(0, l - 1, 1));
        if (l + 1 < L) up(r, l, jj, tr(1, l, 0), tr(1, l, 1), tr(0, l, 0), tr(0, l, 1));
        if (jj == 0) ident(r, 0, tr(1, l - 1, 0), -1.0);
        else { ident(r, 0, tr(1, l - 1, 1), -1.0); ident(r, 0, tr(0, l - 1, 1), -1.0); }
        v.push_back(r);
      }
    }
    return v;
  }
  // y = R x: the couplings between down- and up-going unknowns.
  std::vector<ApplyRow> coupling() const {
    std::vector<ApplyRow> v;
    const int L = P.L;
    for (int l = 0; l + 1 < L; ++l) {
      for (int jj = 2; jj <= 3; ++jj) {
        ApplyRow r = row(tr(0, l, jj - 2));
        if (l >= 1) down(r, l, jj, tr(1, l - 1, 0), tr(1, l - 1, 1));
        up(r, l, jj, tr(1, l, 0), tr(1, l, 1));
        if (jj == 2) ident(r, 0, tr(1, l, 0), -1.0);
        v.push_back(r);
      }
    }
    for (int l = 1; l < L; ++l) {
      for (int jj = 0; jj <= 1; ++jj) {
        ApplyRow r = row(tr(1, l - 1, jj));
        down(r, l, jj, tr(0, l - 1, 0), tr(0, l - 1, 1));
        if (l + 1 < L) up(r, l, jj, tr(0, l, 0), tr(0, l, 1));
        if (jj == 1) ident(r, 0, tr(0, l - 1, 1), -1.0);
        v.push_back(r);
      }
    }
    return v;
  }
  // D^{-1}: step s solves the down-going traces of interface s (top-down
  // sweep) and the up-going traces of interface L-2-s (bottom-up sweep):
  //   y_down[l] = T_down^l y_down[l-1] - r_down[l],   y_up[l-1] = T_up^l y_up[l] - r_up[l-1].
  std::vector<ApplyRow> sweeps() const {
    std::vector<ApplyRow> v;
    const int L = P.L;
    for (int s = 0; s + 1 < L; ++s) {
      const int l = s;
      for (int jj = 2; jj <= 3; ++jj) {
        ApplyRow r = row(tr(0, l, jj - 2));
        if (l >= 1) down(r, l, jj, tr(0, l - 1, 0), tr(0, l - 1, 1));
        ident(r, 1, tr(0, l, jj - 2), -1.0);
        v.push_back(r);
      }
      const int lu = L - 1 - s;
      for (int jj = 0; jj <= 1; ++jj) {
        ApplyRow r = row(tr(1, lu - 1, jj));
        if (lu + 1 < L) up(r, lu, jj, tr(1, lu, 0), tr(1, lu, 1));
        ident(r, 1, tr(1, lu - 1, jj), -1.0);
        v.push_back(r);
      }
    }
    return v;
  }
};

// Tensor-core tables: the same terms with the staged input of each term
// (sign * (x[in1] + x[in2])) deduplicated into keys.
void tc_from(const ApplyRow* rows, int nrows, int nt, std::vector<TcRow>& out, std::vector<TcKey>& keys) {
  std::map<std::tuple<int, int, int>, int> kmap;
  for (int i = 0; i < nrows; ++i) {
    const ApplyRow& a = rows[i];
    TcRow r;
    std::memset(&r, 0, sizeof(r));
    r.out = a.out;
    r.nterms = a.nterms;
    for (int t = 0; t < a.nterms; ++t) {
      const auto k = std::make_tuple(a.t[t].in1, a.t[t].in2, a.t[t].sign > 0 ? 1 : -1);
      auto it = kmap.find(k);
      int idx;
      if (it == kmap.end()) {
        idx = (int)keys.size();
        kmap[k] = idx;
        keys.push_back(TcKey{a.t[t].in1, a.t[t].in2, a.t[t].sign > 0 ? 1.0 : -1.0});
      } else {
        idx = it->second;
      }
      r.t[t] = TcTerm{a.t[t].block * nt, idx};
    }
    r.nid = a.nid;
    for (int e = 0; e < a.nid; ++e) {
      r.id_src[e] = a.id_src[e];
      r.id_trace[e] = a.id_trace[e];
      r.id_sign[e] = a.id_sign[e];
    }
    out.push_back(r);
  }
}

// The one-launch FP32 sweep stages one input per (pair of output traces, term): rows 2g and
// 2g+1 of every step must have the same terms up to their blocks, single input traces and
// identities on the auxiliary vector.
bool sweep_pairs_match(const std::vector<ApplyRow>& sw) {
  if (sw.size() % 4 != 0) return false;
  for (size_t i = 0; i < sw.size(); ++i) {
    const ApplyRow& a = sw[i];
    if (a.nterms > 2) return false;
    for (int t = 0; t < a.nterms; ++t)
      if (a.t[t].in2 >= 0) return false;
    for (int e = 0; e < a.nid; ++e)
      if (a.id_src[e] != 1) return false;
    if (i % 2 == 1) {
      const ApplyRow& b = sw[i - 1];
      if (a.nterms != b.nterms) return false;
      for (int t = 0; t < a.nterms; ++t)
        if (a.t[t].in1 != b.t[t].in1 || a.t[t].sign != b.t[t].sign) return false;
    }
  }
  return true;
}

pt_status full_plan(const pt_params* p, Plan& P) {
  pt_status st = make_plan(p, P);
  if (st != PT_OK) return st;
  if (p->precision == PT_MIXED_TC) {
    P.tc = true;
    P.ldtc = tc_ld(P.nt);
    TableBuilder tb{P};
    auto mv = tb.matvec(), rr = tb.coupling(), sw = tb.sweeps();
    tc_from(mv.data(), (int)mv.size(), P.nt, P.tc_mv, P.tk_mv);
    tc_from(rr.data(), (int)rr.size(), P.nt, P.tc_R, P.tk_R);
    for (int step = 0; step + 1 < P.L; ++step) {
      std::vector<TcKey> k1;
      tc_from(sw.data() + 4 * step, 4, P.nt, P.tc_sw, k1);
      P.tk_sw_off.push_back((int)P.tk_sw.size());
      P.tk_sw_cnt.push_back((int)k1.size());
      P.tk_sw.insert(P.tk_sw.end(), k1.begin(), k1.end());
      P.tc_keys_max = std::max(P.tc_keys_max, (int)k1.size());
    }
    P.tc_keys_max = std::max({P.tc_keys_max, (int)P.tk_mv.size(), (int)P.tk_R.size()});
  }
  return PT_OK;
}

}  // namespace

struct pt_ctx {
  pt_params prm{};
  Plan P;
  Persist d{};
  cudaStream_t stream = nullptr;
  int64_t launches = 0;
  int last_max_it = 0;
  std::vector<double> resid_h;
  // PLR projection task counts per operator table
  int ntask_mv = 0, ntask_R = 0;
  std::vector<int> sw_off, sw_cnt;
  size_t plr_stored = 0;  // complex entries of the compressed representation
  int plr_leaves = 0;
  cd* tbuf = nullptr;     // projection buffer of the current call
  // tensor-core form
  int eA = 0;
  CUtensorMap mapAhi, mapAlo, mapBhi, mapBlo;
  CUtensorMap mapOzA, mapOzX;  // slices of the blocks and of the staged inputs (split restart product)
  CUtensorMap mapBsw;          // staged inputs with the narrower column tile of the sweep steps
  int tc_bn_sw = 0;
  __half* oz_x = nullptr;
  int* oz_f = nullptr;
  int opt_restart = 1;      // PT_OPT_RESTART (PT_MIXED_TC)
  int tc_bn = 0, tc_S = 0;
  __half *tc_bhi = nullptr, *tc_blo = nullptr;
  float *tc_scale = nullptr, *tc_inv = nullptr;
  int opt_layer_group = 0;  // PT_OPT_LAYER_GROUP
  int sweep_terms_max = 0;  // block terms of the longest sweep row
  int opt_local_solve = 0;  // PT_OPT_LOCAL_SOLVE
  int opt_sweep = 0;        // PT_OPT_SWEEP
  int opt_relax = 0;        // PT_OPT_RELAX
  int opt_precond16 = 0;    // PT_OPT_PRECOND_FP16
  int relaxed_matvecs = 0;  // FP32 matvecs of the last solve
  bool sweep_fusable = false;  // sweep tables have the pair layout of the one-launch sweep
  // learned correction
  bool nn_ready = false;    // weights set or trained
  int nn_t = 0;             // Adam steps taken
  int opt_learned = 0;      // PT_OPT_LEARNED
  int learned_used = 0;     // cycles of the last solve that applied the correction
  int last_cycles = 0;      // restart cycles (explicit residuals) of the last solve
  int device = -1;          // the CUDA device current at pt_create
};

static const char* kStatusText[] = {"ok", "invalid argument", "workspace too small", "CUDA error",
                                    "singular local factorization", "GMRES did not converge",
                                    "device-side wait timed out", "non-finite or non-positive data"};

extern "C" const char* pt_status_string(pt_status s) {
  int i = (int)s;
  return (i >= 0 && i < 8) ? kStatusText[i] : "unknown status";
}

extern "C" const char* pt_last_error(void) { return g_last_error.c_str(); }

extern "C" pt_status pt_layer_partition(const pt_params* prm, int32_t* row_start) {
  Plan P;
  pt_status st = full_plan(prm, P);
  if (st != PT_OK) return st;
  if (!row_start) return fail(PT_ERR_ARG, "row_start is NULL");
  for (int l = 0; l < P.L; ++l) row_start[l] = P.layers[l].start;
  row_start[P.L] = P.Nz;
  return PT_OK;
}

extern "C" pt_status pt_workspace_size(const pt_params* prm, size_t* persistent_bytes, size_t* setup_bytes,
                                       size_t* solve_bytes) {
  Plan P;
  pt_status st = full_plan(prm, P);
  if (st != PT_OK) return st;
  size_t pb = 0, sb = 0;
  carve_persist(P, prm, nullptr, &pb);
  carve_solve(P, prm->max_sources, prm->max_krylov, false, nullptr, &sb);
  if (persistent_bytes) *persistent_bytes = pb;
  if (setup_bytes) *setup_bytes = std::max(setup_bytes_of(P), plr_setup_bytes(P));
  if (solve_bytes) *solve_bytes = sb;
  return PT_OK;
}

static pt_status read_status(pt_ctx* c) {
  int st = 0;
  PT_CUDA(cudaMemcpyAsync(&st, c->d.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (st & kErrNumeric) return fail(PT_ERR_NUMERIC, "non-finite or non-positive value met on the device");
  if (st & kErrSingular) return fail(PT_ERR_SINGULAR, "zero pivot in a local factorization");
  if (st & kErrTimeout) return fail(PT_ERR_TIMEOUT, "a device-side wait gave up");
  return PT_OK;
}

// Algorithm 5 on every interface block, then the host-side tables of the
// flattened application: per-block leaf ordinals, the (block, row tile) CSR
// of covering leaves and the projection tasks of each operator table.
static pt_status compress_blocks(pt_ctx* c, void* setup, const std::vector<ApplyRow>& mv,
                                 const std::vector<ApplyRow>& rr, const std::vector<ApplyRow>& sw) {
  const Plan& P = c->P;
  cudaStream_t s = c->stream;
  const int nb = (int)P.plr_blocks.size();
  const int nslots = std::min(nb, kPlrSlots);
  PT_CUDA(cudaMemcpyAsync(c->d.plr_ids, P.plr_blocks.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
  PT_CUDA(launch_plr_compress(P.nt, c->d.blocks, c->d.plr_ids, nb, P.rmax, c->prm.plr_eps, P.oversample,
                              static_cast<cd*>(setup), nslots, c->d.leaves, kPlrCap, c->d.nleaves, c->d.pool,
                              c->d.status, s));
  std::vector<int> nl(nb);
  std::vector<PlrLeaf> lv((size_t)nb * kPlrCap);
  PT_CUDA(cudaMemcpyAsync(nl.data(), c->d.nleaves, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
  PT_CUDA(cudaMemcpyAsync(lv.data(), c->d.leaves, lv.size() * sizeof(PlrLeaf), cudaMemcpyDeviceToHost, s));
  PT_CUDA(cudaStreamSynchronize(s));
  pt_status st = read_status(c);
  if (st != PT_OK) return st;
  std::vector<int> bmap((size_t)P.L * 16, -1);
  for (int b = 0; b < nb; ++b) bmap[P.plr_blocks[b]] = b;
  std::vector<int> lr((size_t)nb * kPlrCap, 0);
  std::vector<std::vector<int>> bucket((size_t)P.L * 16 * P.ntiles);
  c->plr_stored = 0;
  c->plr_leaves = 0;
  for (int b = 0; b < nb; ++b) {
    int ord = 0;
    for (int i = 0; i < nl[b]; ++i) {
      const PlrLeaf& f = lv[(size_t)b * kPlrCap + i];
      const int li = b * kPlrCap + i;
      if (f.kind == 1) lr[li] = ord++;
      c->plr_stored += f.kind == 1 ? (size_t)f.rank * (f.m + f.n) : (size_t)f.m * f.n;
      c->plr_leaves++;
      for (int t = f.r0 / 32; t <= (f.r0 + f.m - 1) / 32; ++t)
        bucket[(size_t)P.plr_blocks[b] * P.ntiles + t].push_back(li);
    }
  }
  std::vector<int> tptr(bucket.size() + 1, 0), tleaf;
  for (size_t q = 0; q < bucket.size(); ++q) {
    tptr[q] = (int)tleaf.size();
    tleaf.insert(tleaf.end(), bucket[q].begin(), bucket[q].end());
  }
  tptr[bucket.size()] = (int)tleaf.size();
  auto build = [&](const ApplyRow* rows, int nrows, std::vector<PlrTask>& tasks, std::vector<int>& tbase) {
    tbase.assign((size_t)nrows * 4, 0);
    for (int r = 0; r < nrows; ++r)
      for (int t = 0; t < rows[r].nterms; ++t) {
        const int b = bmap[rows[r].t[t].block];
        tbase[r * 4 + t] = (int)tasks.size();
        for (int i = 0; i < nl[b]; ++i)
          if (lv[(size_t)b * kPlrCap + i].kind == 1) tasks.push_back(PlrTask{r, t, b * kPlrCap + i});
      }
  };
  std::vector<PlrTask> tmv, trr, tsw;
  std::vector<int> bmv, brr, bsw;
  build(mv.data(), (int)mv.size(), tmv, bmv);
  build(rr.data(), (int)rr.size(), trr, brr);
  c->sw_off.clear();
  c->sw_cnt.clear();
  for (int step = 0; step + 1 < P.L; ++step) {
    std::vector<PlrTask> t1;
    std::vector<int> b1;
    build(sw.data() + 4 * step, 4, t1, b1);
    c->sw_off.push_back((int)tsw.size());
    c->sw_cnt.push_back((int)t1.size());
    for (int& v : b1) v += 0;  // task indices are relative to the step's own task list
    tsw.insert(tsw.end(), t1.begin(), t1.end());
    bsw.insert(bsw.end(), b1.begin(), b1.end());
  }
  if (tmv.size() > P.plr_task_cap || trr.size() > P.plr_task_cap || tsw.size() > P.plr_task_cap ||
      tleaf.size() > (size_t)nb * kPlrCap * P.ntiles)
    return fail(PT_ERR_WORKSPACE, "PLR tables exceed their bounds");
  c->ntask_mv = (int)tmv.size();
  c->ntask_R = (int)trr.size();
  PT_CUDA(cudaMemcpyAsync(c->d.lr_ord, lr.data(), lr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tile_ptr, tptr.data(), tptr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!tleaf.empty())
    PT_CUDA(cudaMemcpyAsync(c->d.tile_leaf, tleaf.data(), tleaf.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!tmv.empty()) PT_CUDA(cudaMemcpyAsync(c->d.task_mv, tmv.data(), tmv.size() * sizeof(PlrTask), cudaMemcpyHostToDevice, s));
  if (!trr.empty()) PT_CUDA(cudaMemcpyAsync(c->d.task_R, trr.data(), trr.size() * sizeof(PlrTask), cudaMemcpyHostToDevice, s));
  if (!tsw.empty()) PT_CUDA(cudaMemcpyAsync(c->d.task_sw, tsw.data(), tsw.size() * sizeof(PlrTask), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tbase_mv, bmv.data(), bmv.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tbase_R, brr.data(), brr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tbase_sw, bsw.data(), bsw.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (c->d.pool32) PT_CUDA(launch_pool_to_fp32(c->d.pool, c->d.pool32, (size_t)nb * P.nt * P.nt, s));
  PT_CUDA(cudaStreamSynchronize(s));
  return PT_OK;
}

// FP16 [Br Bi] copies of the blocks with one power-of-two scale (max entry in
// [2^9, 2^10)), the tensor-core tables, and the tensor maps of the block rows.
static pt_status prepare_tc(pt_ctx* c) {
  const Plan& P = c->P;
  cudaStream_t s = c->stream;
  const size_t nb = (size_t)P.L * 16 * P.nt * P.nt;
  PT_CUDA(cudaMemsetAsync(c->d.tc_max, 0, sizeof(unsigned long long), s));
  PT_CUDA(launch_max_abs(c->d.blocks, nb, c->d.tc_max, s));
  unsigned long long bits = 0;
  PT_CUDA(cudaMemcpyAsync(&bits, c->d.tc_max, sizeof(bits), cudaMemcpyDeviceToHost, s));
  PT_CUDA(cudaStreamSynchronize(s));
  double mx;
  std::memcpy(&mx, &bits, sizeof(mx));
  int ex = 0;
  if (mx > 0) std::frexp(mx, &ex);
  c->eA = 10 - ex;
  PT_CUDA(launch_tc_blocks(c->d.blocks, (size_t)P.L * 16 * P.nt, P.nt, P.ldtc, std::ldexp(1.0, c->eA), c->d.tc_ahi,
                           c->d.tc_alo, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tcr_mv, P.tc_mv.data(), P.tc_mv.size() * sizeof(TcRow), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tcr_R, P.tc_R.data(), P.tc_R.size() * sizeof(TcRow), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tcr_sw, P.tc_sw.data(), P.tc_sw.size() * sizeof(TcRow), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tck_mv, P.tk_mv.data(), P.tk_mv.size() * sizeof(TcKey), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tck_R, P.tk_R.data(), P.tk_R.size() * sizeof(TcKey), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemcpyAsync(c->d.tck_sw, P.tk_sw.data(), P.tk_sw.size() * sizeof(TcKey), cudaMemcpyHostToDevice, s));
  const size_t rowsA = (size_t)P.L * 16 * P.nt;
  if (!tc_make_map(&c->mapAhi, c->d.tc_ahi, rowsA, P.ldtc, P.ldtc, 128) ||
      !tc_make_map(&c->mapAlo, c->d.tc_alo, rowsA, P.ldtc, P.ldtc, 128))
    return fail(PT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the block rows");
  // slices of the blocks for the split restart product (exact tensor-core accumulation)
  PT_CUDA(launch_oz_blocks(c->d.blocks, rowsA, P.nt, P.ldtc, c->d.oz_a, c->d.oz_e, s));
  if (!tc_make_map(&c->mapOzA, c->d.oz_a, (size_t)oz_slices() * rowsA, P.ldtc, P.ldtc, 128))
    return fail(PT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the block slices");
  PT_CUDA(cudaStreamSynchronize(s));
  return PT_OK;
}

extern "C" pt_status pt_create(const pt_params* prm, const double* c_ext, void* persistent, size_t persistent_bytes,
                               void* setup, size_t setup_bytes, void* stream, pt_ctx** out) {
  if (!out) return fail(PT_ERR_ARG, "out is NULL");
  *out = nullptr;
  Plan P;
  pt_status st = full_plan(prm, P);
  if (st != PT_OK) return st;
  if (!c_ext || !persistent || !setup) return fail(PT_ERR_ARG, "NULL device pointer");
  if (((uintptr_t)persistent % kAlign) || ((uintptr_t)setup % kAlign))
    return fail(PT_ERR_ARG, "workspaces must be 256-byte aligned");
  size_t need_p = 0;
  carve_persist(P, prm, nullptr, &need_p);
  if (persistent_bytes < need_p || setup_bytes < std::max(setup_bytes_of(P), plr_setup_bytes(P)))
    return fail(PT_ERR_WORKSPACE, "persistent or setup workspace too small");
  pt_ctx* c = new (std::nothrow) pt_ctx();
  if (!c) return fail(PT_ERR_ARG, "host allocation failed");
  c->prm = *prm;
  c->prm.layer_rows = nullptr;  // the partition lives in the plan; the caller's array is not kept
  c->P = P;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return fail(PT_ERR_CUDA, "cudaGetDevice"); }
  c->stream = static_cast<cudaStream_t>(stream);
  c->d = carve_persist(P, prm, persistent, nullptr);
  if (c->d.chunk_T) c->opt_local_solve = 4;  // mixed FP32: chunked local solves by default
  if (prm->precision == PT_MIXED_FP32) c->opt_relax = 1;
  // FP16 preconditioner blocks are an option: on the 511 x 1023, L = 16 workload they cost one
  // more GMRES iteration than the complex64 ones, which outweighs the halved sweep stream
  auto bail = [&](pt_status s) { delete c; return s; };
  cudaStream_t s = c->stream;
  const Geometry& g = P.g;
  if (cudaMemsetAsync(c->d.status, 0, 64 * sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(c->d.layers, P.layers.data(), P.L * sizeof(LayerInfo), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->d.tasks, P.tasks.data(), P.tasks.size() * sizeof(ExtractTask), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return bail(fail(PT_ERR_CUDA, "copying tables"));
  TableBuilder tb{P};
  auto mv = tb.matvec(), rr = tb.coupling(), sw = tb.sweeps();
  c->sweep_terms_max = 0;
  for (const ApplyRow& ar : sw) c->sweep_terms_max = std::max(c->sweep_terms_max, ar.nterms);
  c->sweep_fusable = sweep_pairs_match(sw);
  if (cudaMemcpyAsync(c->d.tab_matvec, mv.data(), mv.size() * sizeof(ApplyRow), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(c->d.tab_R, rr.data(), rr.size() * sizeof(ApplyRow), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(c->d.tab_sweep, sw.data(), sw.size() * sizeof(ApplyRow), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return bail(fail(PT_ERR_CUDA, "copying operator tables"));
  // Algorithm 1
  if (launch_check_medium(c_ext, (size_t)P.Nz * P.nt, c->d.status, s) != cudaSuccess) return bail(fail(PT_ERR_CUDA, "check"));
  if (cudaMemsetAsync(c->d.blocks, 0, (size_t)P.L * 16 * P.nt * P.nt * sizeof(cd), s) != cudaSuccess ||
      cudaMemcpyAsync(c->d.m_ext, c_ext, (size_t)P.Nz * P.nt * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return bail(fail(PT_ERR_CUDA, "initialising the block storage"));
  st = read_status(c);
  if (st != PT_OK) return bail(st);
  cudaError_t e = launch_coef(g, c->d.layers, c_ext, c->d.W, c->d.E, s);
  if (e == cudaSuccess) e = launch_factor(g, c->d.layers, P.nloc_max, c_ext, c->d.Sinv, c->d.status, s);
  const int nslots = std::min<int>((int)P.tasks.size(), kExtractSlots);
  if (e == cudaSuccess)
    e = launch_extract(g, c->d.layers, c->d.tasks, (int)P.tasks.size(), nslots, P.nloc_max, c->d.Sinv, c->d.W,
                       c->d.E, static_cast<cd*>(setup), setup_slot_elems(P), c->d.blocks, s);
  if (e == cudaSuccess && c->d.blocks_hi)
    e = launch_split_blocks(c->d.blocks, P.nt, P.ld32, (size_t)P.L * 16 * P.nt, c->d.blocks_hi, c->d.blocks_lo, s);
  if (e == cudaSuccess && c->d.blocks_h16)
    e = launch_blocks_h16(c->d.blocks, P.nt, P.ld32, (size_t)P.L * 16 * P.nt, c->d.blocks_h16, c->d.bscale, s);
  if (e == cudaSuccess && c->d.sinv_hi) e = launch_split_sinv(c->d.Sinv, P.sinv_elems, c->d.sinv_hi, c->d.sinv_lo, s);
  if (e == cudaSuccess && c->d.w_hi) e = launch_split_sinv(c->d.W, P.coef_elems, c->d.w_hi, c->d.w_lo, s);
  if (e == cudaSuccess && c->d.e_hi) e = launch_split_sinv(c->d.E, P.coef_elems, c->d.e_hi, c->d.e_lo, s);
  if (e == cudaSuccess && c->d.chunk_T) {  // after the extraction: it reuses the setup scratch
    e = cudaMemsetAsync(c->d.chunk_T, 0, (size_t)P.L * (P.kr + P.kv) * 3 * P.nloc_max * P.nloc_max * sizeof(cf), s);
    if (e == cudaSuccess)
      e = launch_chunk_transfer(g, c->d.layers, c->d.Sinv, c->d.W, c->d.E, P.kr, P.nloc_max, static_cast<cd*>(setup),
                              c->d.chunk_T, s);
    if (e == cudaSuccess)
      e = launch_chunk_transfer(g, c->d.layers, c->d.Sinv, c->d.W, c->d.E, P.kv, P.nloc_max,
                                static_cast<cd*>(setup),
                                c->d.chunk_T + (size_t)P.L * P.kr * 3 * P.nloc_max * P.nloc_max, s);
  }
  if (e != cudaSuccess) return bail(fail(PT_ERR_CUDA, std::string("offline launch: ") + cudaGetErrorString(e)));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(fail(PT_ERR_CUDA, std::string("offline phase: ") + cudaGetErrorString(e)));
  st = read_status(c);
  if (st != PT_OK) return bail(st);
  if (P.plr) {
    st = compress_blocks(c, setup, mv, rr, sw);
    if (st != PT_OK) return bail(st);
  }
  if (P.tc) {
    st = prepare_tc(c);
    if (st != PT_OK) return bail(st);
  }
  *out = c;
  return PT_OK;
}

extern "C" void pt_destroy(pt_ctx* ctx) { delete ctx; }

// Point the context at this call's scratch: PLR projections and, in the
// tensor-core form, the staged operands and their tensor maps.
static pt_status bind_call(pt_ctx* c, const SolveBufs& B, int S) {
  c->tbuf = B.tbuf;
  if (!c->P.tc) return PT_OK;
  c->tc_bhi = B.tc_bhi;
  c->tc_blo = B.tc_blo;
  c->tc_scale = B.tc_scale;
  c->tc_inv = B.tc_inv;
  const int two_s = 2 * S;
  c->tc_bn = two_s <= 64 ? 64 : (two_s <= 128 ? 128 : 256);
  // a sweep step has only four output traces: narrower column tiles give it more CTAs
  c->tc_bn_sw = std::min(c->tc_bn, 128);
  const size_t rows = (size_t)c->P.tc_keys_max * two_s;
  if (!tc_make_map(&c->mapBhi, B.tc_bhi, rows, c->P.ldtc, c->P.ldtc, c->tc_bn) ||
      !tc_make_map(&c->mapBlo, B.tc_blo, rows, c->P.ldtc, c->P.ldtc, c->tc_bn))
    return fail(PT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the staged operands");
  if (!tc_make_map(&c->mapBsw, B.tc_bhi, rows, c->P.ldtc, c->P.ldtc, c->tc_bn_sw))
    return fail(PT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the staged operands of the sweeps");
  c->oz_x = B.oz_x;
  c->oz_f = B.oz_f;
  if (!tc_make_map(&c->mapOzX, B.oz_x, (size_t)oz_slices() * c->P.tk_mv.size() * two_s, c->P.ldtc, c->P.ldtc,
                   oz_bn()))
    return fail(PT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the staged input slices");
  c->tc_S = S;
  return PT_OK;
}

// ---- online building blocks ------------------------------------------------
namespace {

enum { kModeFP64 = 0, kModeFP32 = 1, kModeDF = 2, kModeTC1 = 3, kModeTC3 = 4, kModeH16 = 5 };

bool mixed(const pt_ctx* c) { return c->prm.precision == PT_MIXED_FP32 || c->prm.precision == PT_MIXED_TC; }
bool tcmode(const pt_ctx* c) { return c->prm.precision == PT_MIXED_TC; }

struct OpRef {
  const ApplyRow* table;
  int nrows;
  const PlrTask* tasks;  // PLR projection tasks of this table (null without PLR)
  int ntasks;
  const int* tbase;
  const TcRow* tcr;      // tensor-core rows and staged-input keys (PT_MIXED_TC)
  const TcKey* tck;
  int nkeys;
  bool sweep = false;    // one sweep step (four output traces)
};

// Dense apply in the given arithmetic mode, or the PLR apply when the context
// compresses its blocks and the caller asks for the working representation.
cudaError_t apply(pt_ctx* c, int mode, const OpRef& op, int S, const cd* x, const cd* aux, cd* y, int rows_per_cta,
                  double alpha, double beta, bool working) {
  const Plan& P = c->P;
  if (mode == kModeTC1 || mode == kModeTC3) {
    // staged inputs with the per-source scales set by tc_scale(), then the tensor-core products
    const int npass = mode == kModeTC3 ? 3 : 1;
    c->launches += 2;
    cudaError_t e = launch_tc_stage(op.tck, op.nkeys, x, P.nt, P.T4, S, P.ldtc, c->tc_scale, c->tc_bhi,
                                    npass == 3 ? c->tc_blo : nullptr, c->stream);
    if (e != cudaSuccess) return e;
    if (op.sweep && npass == 1)
      return launch_tc_apply(c->tc_bn_sw, c->mapAhi, c->mapAlo, c->mapBsw, c->mapBlo, op.tcr, op.nrows, P.nt, P.T4,
                             S, npass, c->tc_inv, x, aux, y, alpha, beta, c->d.status, c->stream);
    return launch_tc_apply(c->tc_bn, c->mapAhi, c->mapAlo, c->mapBhi, c->mapBlo, op.tcr, op.nrows, P.nt, P.T4, S,
                           npass, c->tc_inv, x, aux, y, alpha, beta, c->d.status, c->stream);
  }
  if (working && P.plr) {
    const bool fp32 = mode == kModeFP32;
    c->launches += (op.ntasks > 0 ? 2 : 1);
    return launch_plr_apply(fp32, P.nt, P.T4, fp32 ? P.ld32 : P.nt, op.table, op.nrows,
                            fp32 ? static_cast<const void*>(c->d.blocks_hi) : static_cast<const void*>(c->d.blocks),
                            fp32 ? static_cast<const void*>(c->d.pool32) : static_cast<const void*>(c->d.pool),
                            c->d.leaves, op.tasks, op.ntasks, c->d.tile_ptr, c->d.tile_leaf, op.tbase, c->d.lr_ord,
                            c->tbuf, P.rmax, x, aux, y, S, alpha, beta, c->stream);
  }
  c->launches++;
  if (mode == kModeFP64)
    return launch_apply_mode(kModeFP64, P.nt, P.nt, P.T4, op.table, op.nrows, c->d.blocks, nullptr, x, aux, y, S,
                             rows_per_cta, alpha, beta, c->stream);
  if (mode == kModeFP32 && rows_per_cta == kApplyRowsSweep && c->sweep_terms_max <= 2) {
    // sweep steps: one row per warp with both block rows in flight
    cudaError_t e = cudaSuccess;
    if (launch_apply_f32_rows(P.nt, P.ld32, P.T4, op.table, op.nrows, c->d.blocks_hi, x, aux, y, S, alpha, beta,
                              c->stream, &e))
      return e;
  }
  if ((mode == kModeFP32 || mode == kModeDF || (mode == kModeH16 && c->d.blocks_h16)) && c->d.xprep && !P.plr) {
    // inputs converted once, FP32 staging, FP64 epilogue on one thread per row
    c->launches++;
    cudaError_t e = launch_prep_inputs(x, S * P.T4, P.nt, P.ld32, mode == kModeDF, c->d.xprep, c->stream);
    if (e != cudaSuccess) return e;
    if (mode == kModeH16)  // FP16 blocks with row scales (kernel mode 3)
      return launch_apply_lowp(3, P.nt, P.ld32, P.T4, op.table, op.nrows, c->d.blocks_h16, c->d.bscale, c->d.xprep, x,
                               aux, y, S, rows_per_cta, alpha, beta, c->stream);
    return launch_apply_lowp(mode, P.nt, P.ld32, P.T4, op.table, op.nrows, c->d.blocks_hi, c->d.blocks_lo,
                             c->d.xprep, x, aux, y, S, rows_per_cta, alpha, beta, c->stream);
  }
  if (mode == kModeH16) mode = kModeFP32;  // no FP16 copies: the FP32 ones
  return launch_apply_mode(mode, P.nt, P.ld32, P.T4, op.table, op.nrows, c->d.blocks_hi, c->d.blocks_lo, x, aux, y,
                           S, rows_per_cta, alpha, beta, c->stream);
}

OpRef op_matvec(pt_ctx* c) {
  return OpRef{c->d.tab_matvec, c->P.T4, c->d.task_mv, c->ntask_mv, c->d.tbase_mv, c->d.tcr_mv, c->d.tck_mv,
               (int)c->P.tk_mv.size()};
}
OpRef op_R(pt_ctx* c) {
  return OpRef{c->d.tab_R, c->P.T4, c->d.task_R, c->ntask_R, c->d.tbase_R, c->d.tcr_R, c->d.tck_R,
               (int)c->P.tk_R.size()};
}
OpRef op_sweep(pt_ctx* c, int step) {
  OpRef o{c->d.tab_sweep + 4 * step, 4, nullptr, 0, nullptr, nullptr, nullptr, 0, true};
  if (c->P.plr) {
    o.tasks = c->d.task_sw + c->sw_off[step];
    o.ntasks = c->sw_cnt[step];
    o.tbase = c->d.tbase_sw + 16 * step;
  }
  if (c->P.tc) {
    o.tcr = c->d.tcr_sw + 4 * step;
    o.tck = c->d.tck_sw + c->P.tk_sw_off[step];
    o.nkeys = c->P.tk_sw_cnt[step];
  }
  return o;
}

// Per-source FP16 scales of a tensor-core apply, from the vector `ref`.
cudaError_t tc_scale(pt_ctx* c, int S, const cd* ref) {
  c->launches++;
  return launch_tc_scale(ref, c->P.N, S, c->eA, c->tc_scale, c->tc_inv, c->stream);
}

// y = P M x.  exact: dense FP64 blocks (the true residual and the public
// matvec); otherwise the working form: PLR blocks in FP64 when compressed,
// else double-float (mixed) or FP64 dense blocks.
cudaError_t do_matvec(pt_ctx* c, int S, const cd* x, cd* y, bool exact = true) {
  if (exact) return apply(c, kModeFP64, op_matvec(c), S, x, nullptr, y, kApplyRowsWide, 1.0, 0.0, false);
  if (tcmode(c)) {
    cudaError_t e = tc_scale(c, S, x);
    if (e != cudaSuccess) return e;
    return apply(c, kModeTC3, op_matvec(c), S, x, nullptr, y, kApplyRowsWide, 1.0, 0.0, true);
  }
  const int mode = (c->P.plr || !mixed(c)) ? kModeFP64 : kModeDF;
  return apply(c, mode, op_matvec(c), S, x, nullptr, y, kApplyRowsWide, 1.0, 0.0, true);
}

// y = P M x in the arithmetic of the explicit residual between restart cycles (iterative
// refinement): FP64 blocks in PT_FP64 and with compressed blocks; in the mixed forms the
// double-float product (~1e-14) on the FP32 pipes (the FP64 pipe bounds an FP64 product at
// about twice its time), which in PT_MIXED_TC also corrects the ~1e-5 tensor-core matvec of
// the inner cycles
cudaError_t do_restart_matvec(pt_ctx* c, int S, const cd* x, cd* y) {
  if (tcmode(c) && c->opt_restart == 1) {
    // split products on the tensor cores (exact FP32 accumulation per 512-long segment, ~1e-10)
    const Plan& P = c->P;
    const int nk = (int)P.tk_mv.size();
    c->launches += 3;
    cudaError_t e = launch_oz_source_exp(x, P.N, S, c->oz_f, c->stream);
    if (e == cudaSuccess)
      e = launch_oz_stage(c->d.tck_mv, nk, x, P.nt, P.T4, S, P.ldtc, c->oz_f, (size_t)nk * 2 * S, c->oz_x, c->stream);
    if (e == cudaSuccess)
      e = launch_oz_apply(c->mapOzA, c->mapOzX, c->d.tcr_mv, P.T4, P.nt, P.T4, S, (int)((size_t)P.L * 16 * P.nt),
                          nk * 2 * S, c->d.oz_e, c->oz_f, x, nullptr, y, 1.0, 0.0, c->d.status, c->stream);
    return e;
  }
  if (mixed(c) && !c->P.plr) return apply(c, kModeDF, op_matvec(c), S, x, nullptr, y, kApplyRowsWide, 1.0, 0.0, false);
  return do_matvec(c, S, x, y);
}

// y = alpha R x + beta aux
cudaError_t do_R(pt_ctx* c, int S, const cd* x, cd* y, int mode, double alpha = 1.0, double beta = 0.0,
                 const cd* aux = nullptr, bool working = false) {
  if (mode == kModeTC1 || mode == kModeTC3) {
    cudaError_t e = tc_scale(c, S, x);
    if (e != cudaSuccess) return e;
  }
  return apply(c, mode, op_R(c), S, x, aux, y, kApplyRowsWide, alpha, beta, working);
}

// y = D^{-1} r (one launch per sweep step, down and up sweeps together); y must not alias r.
cudaError_t do_Dinv(pt_ctx* c, int S, const cd* r, cd* y, int mode, bool working = false) {
  const int steps = c->P.L - 1;
  if (mode == kModeTC1 || mode == kModeTC3) {
    // one scale per source for the whole sweep, from the right-hand side
    cudaError_t e = tc_scale(c, S, r);
    if (e != cudaSuccess) return e;
  }
  if ((mode == kModeFP32 || mode == kModeH16) && !c->P.plr && c->sweep_fusable && c->opt_sweep == 0 &&
      !g_shared_gpu) {
    // all steps in one cooperative launch (the counter reset is the second operation)
    cudaError_t e = cudaSuccess;
    const bool h16 = mode == kModeH16 && c->d.blocks_h16;
    if (c->d.sweep_y32 &&
        launch_sweep_f32(c->P.nt, c->P.ld32, c->P.T4, steps, c->d.tab_sweep,
                         h16 ? static_cast<const void*>(c->d.blocks_h16) : static_cast<const void*>(c->d.blocks_hi),
                         h16 ? c->d.bscale : nullptr, r, y, c->d.sweep_y32, S, c->d.sweep_bar, c->d.status,
                         c->stream, &e)) {
      c->launches += 2;
      return e;
    }
  }
  for (int s = 0; s < steps; ++s) {
    cudaError_t e = apply(c, mode, op_sweep(c, s), S, y, r, y, kApplyRowsSweep, 1.0, 0.0, working);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Algorithm 4: z = D^{-1} r; repeat n_it - 1 times z = D^{-1}(r - R z).
// Mixed form: FP32 blocks (the preconditioner only has to be approximate in flexible GMRES).
// the arithmetic of the preconditioner's products: FP16 blocks when PT_OPT_PRECOND_FP16 is set
// (mixed FP32 form), otherwise complex64 blocks in the mixed FP32 form, the tensor cores, or FP64
int precond_mode(const pt_ctx* c) {
  if (tcmode(c)) return kModeTC1;
  if (!mixed(c)) return kModeFP64;
  return (c->opt_precond16 && c->d.blocks_h16) ? kModeH16 : kModeFP32;
}

cudaError_t do_precond(pt_ctx* c, int S, const cd* r, cd* z, cd* tmp1, cd* /*tmp2*/) {
  const int mode = precond_mode(c);
  cudaError_t e = do_Dinv(c, S, r, z, mode, true);
  for (int it = 1; it < c->prm.gs_iters && e == cudaSuccess; ++it) {
    e = do_R(c, S, z, tmp1, mode, -1.0, 1.0, r, true);  // tmp1 = r - R z
    if (e == cudaSuccess) e = do_Dinv(c, S, tmp1, z, mode, true);
  }
  return e;
}

cudaError_t do_layer_solve(pt_ctx* c, int mode, int S, const cd* f, const cd* xtr, cd* out, const SolveBufs& B) {
  c->launches++;
  const Plan& P = c->P;
  if (tcmode(c)) {  // many sources: FP32 local solves, one Sinv read per group of sources
    if (!c->d.sinv_hi || !c->d.w_hi || !c->d.e_hi) return cudaErrorInvalidValue;
    return launch_layer_solve_batch(mode, P.g, c->d.layers, P.nloc_max, c->d.sinv_hi, c->d.w_hi, c->d.e_hi, f, xtr,
                                    B.Y, out, B.nzflag, S, c->opt_layer_group, c->stream);
  }
  if (mixed(c)) {
    if (!c->d.sinv_hi || !c->d.w_hi || !c->d.e_hi) return cudaErrorInvalidValue;  // never launch on missing factors
    if (c->opt_local_solve == 4 && c->d.chunk_T && B.chunk_bnd && B.f32) {  // FP32, chunked along x
      const int K = mode == 0 ? P.kr : P.kv;
      const cf* Tm = c->d.chunk_T + (mode == 0 ? 0 : (size_t)P.L * P.kr * 3 * P.nloc_max * P.nloc_max);
      // conversions (sources; for the volume also the traces and the result), phase 1 (K > 1),
      // propagation, phase 3; one of them is counted on entry
      c->launches += (mode == 1 ? 3 : 1) + (K > 1 ? 1 : 0) + 2 - 1;
      cudaError_t e = launch_to_c64(f, (size_t)S * P.Nz * P.nt, B.f32, c->stream);
      if (e != cudaSuccess) return e;
      return launch_layer_solve_chunked(mode, P.g, c->d.layers, P.nloc_max, K, Tm, c->d.sinv_hi, c->d.w_hi,
                                        c->d.e_hi, B.f32, xtr, B.tr32, B.Y, (size_t)P.nt * P.nloc_max, out, B.vol32,
                                        B.nzflag, B.chunk_bnd, S, c->d.status, c->stream);
    }
    if (c->opt_local_solve != 1)  // FP32 on a cluster of 4 (0) or 8 (3) CTAs, or one CTA (2), per (layer, source)
      return launch_layer_solve_f32(mode, P.g, c->d.layers, P.nloc_max, c->d.sinv_hi, c->d.w_hi, c->d.e_hi, f, xtr,
                                    B.Y, (size_t)P.nt * P.nloc_max, out, B.nzflag, B.nzfirst, S, c->d.status,
                                    c->opt_local_solve == 0 ? 4 : (c->opt_local_solve == 3 ? 8 : 1), c->stream);
    return launch_layer_solve_df(mode, P.g, c->d.layers, c->d.sinv_hi, c->d.sinv_lo, c->d.w_hi, c->d.w_lo, c->d.e_hi,
                                 c->d.e_lo, f, xtr, B.Y, (size_t)P.nt * P.nloc_max, out, B.nzflag, S, c->stream);
  }
  return launch_layer_solve2(mode, false, P.g, c->d.layers, c->d.Sinv, nullptr, nullptr, c->d.W, c->d.E, f, xtr,
                             B.Y, (size_t)P.nt * P.nloc_max, out, B.nzflag, S, c->stream);
}

cudaError_t do_rhs(pt_ctx* c, int S, const cd* f, cd* b, const SolveBufs& B) {
  c->launches++;
  cudaError_t e = launch_layer_nonzero(c->P.g, c->d.layers, f, B.nzflag, B.nzfirst, S, c->stream);
  if (e != cudaSuccess) return e;
  return do_layer_solve(c, 0, S, f, nullptr, b, B);
}

pt_status check_solve_args(pt_ctx* c, int nsrc, void* scratch, size_t scratch_bytes, size_t need) {
  if (!c) return fail(PT_ERR_ARG, "ctx is NULL");
  if (nsrc < 1 || nsrc > c->prm.max_sources) return fail(PT_ERR_ARG, "nsrc out of range (1..max_sources)");
  if (!scratch) return fail(PT_ERR_ARG, "scratch is NULL");
  if ((uintptr_t)scratch % kAlign) return fail(PT_ERR_ARG, "scratch must be 256-byte aligned");
  if (scratch_bytes < need) return fail(PT_ERR_WORKSPACE, "scratch too small");
  return PT_OK;
}

}  // namespace

extern "C" pt_status pt_apply_matvec(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y) {
  if (!ctx || !x || !y || nsrc < 1 || nsrc > ctx->prm.max_sources) return fail(PT_ERR_ARG, "bad arguments");
  PT_CUDA(do_matvec(ctx, nsrc, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y)));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_apply(pt_ctx* ctx, int32_t which, int32_t working, int32_t nsrc, const pt_c128* x,
                              pt_c128* y, void* scratch, size_t scratch_bytes) {
  if (!ctx || !x || !y || x == y || which < 0 || which > 3) return fail(PT_ERR_ARG, "bad arguments");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  st = bind_call(ctx, B, nsrc);
  if (st != PT_OK) return st;
  const cd* xd = reinterpret_cast<const cd*>(x);
  cd* yd = reinterpret_cast<cd*>(y);
  const bool w = working != 0;
  if (which == 0) {
    PT_CUDA(do_matvec(ctx, nsrc, xd, yd, !w));
  } else if (which == 3) {
    PT_CUDA(do_restart_matvec(ctx, nsrc, xd, yd));
  } else {
    const int mode = w ? precond_mode(ctx) : kModeFP64;
    if (which == 1) PT_CUDA(do_R(ctx, nsrc, xd, yd, mode, 1.0, 0.0, nullptr, w));
    else PT_CUDA(do_Dinv(ctx, nsrc, xd, yd, mode, w));
  }
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_volume_residual(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, const pt_c128* u,
                                        double* relres, void* scratch, size_t scratch_bytes) {
  if (!ctx || !f || !u || !relres) return fail(PT_ERR_ARG, "bad arguments");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  PT_CUDA(launch_volume_residual(ctx->P.g, ctx->d.m_ext, reinterpret_cast<const cd*>(f),
                                 reinterpret_cast<const cd*>(u), nsrc, B.vres, ctx->stream));
  PT_CUDA(cudaMemcpyAsync(relres, B.vres, nsrc * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_set_option(pt_ctx* ctx, int32_t option, int32_t value) {
  if (!ctx) return fail(PT_ERR_ARG, "ctx is NULL");
  if (option == PT_OPT_LEARNED) {
    if (value != 0 && value != 1) return fail(PT_ERR_ARG, "PT_OPT_LEARNED must be 0 or 1");
    if (value == 1 && !ctx->P.learned) return fail(PT_ERR_ARG, "context created with learned = 0");
    if (value == 1 && !ctx->nn_ready) return fail(PT_ERR_ARG, "no correction weights set or trained");
    ctx->opt_learned = value;
    return PT_OK;
  }
  if (option == PT_OPT_LOCAL_SOLVE) {
    if (value < 0 || value > 4) return fail(PT_ERR_ARG, "PT_OPT_LOCAL_SOLVE must be 0, 1, 2, 3 or 4");
    if (value == 4 && !ctx->d.chunk_T) return fail(PT_ERR_ARG, "chunked local solves need PT_MIXED_FP32");
    ctx->opt_local_solve = value;
    return PT_OK;
  }
  if (option == PT_OPT_PRECOND_FP16) {
    if (value != 0 && value != 1) return fail(PT_ERR_ARG, "PT_OPT_PRECOND_FP16 must be 0 or 1");
    if (value == 1 && !ctx->d.blocks_h16) return fail(PT_ERR_ARG, "FP16 preconditioner blocks need PT_MIXED_FP32, plr = 0");
    ctx->opt_precond16 = value;
    return PT_OK;
  }
  if (option == PT_OPT_RESTART) {
    if (value != 0 && value != 1) return fail(PT_ERR_ARG, "PT_OPT_RESTART must be 0 or 1");
    if (!tcmode(ctx)) return fail(PT_ERR_ARG, "PT_OPT_RESTART needs PT_MIXED_TC");
    ctx->opt_restart = value;
    return PT_OK;
  }
  if (option == PT_OPT_RELAX) {
    if (value != 0 && value != 1) return fail(PT_ERR_ARG, "PT_OPT_RELAX must be 0 or 1");
    if (value == 1 && ctx->prm.precision != PT_MIXED_FP32) return fail(PT_ERR_ARG, "PT_OPT_RELAX needs PT_MIXED_FP32");
    ctx->opt_relax = value;
    return PT_OK;
  }
  if (option == PT_OPT_SWEEP) {
    if (value != 0 && value != 1) return fail(PT_ERR_ARG, "PT_OPT_SWEEP must be 0 or 1");
    ctx->opt_sweep = value;
    return PT_OK;
  }
  if (option == PT_OPT_LAYER_GROUP) {
    if (value != 0 && value != 8 && value != 16 && value != 32) return fail(PT_ERR_ARG, "layer group must be 0, 8, 16 or 32");
    ctx->opt_layer_group = value;
    return PT_OK;
  }
  return fail(PT_ERR_ARG, "unknown option");
}

// ---- learned correction of the preconditioner ---------------------------------
namespace {

// z (+)= N_theta(v) for S permuted residuals, nn_cs sources at a time
cudaError_t do_correction(pt_ctx* c, int S, const cd* v, cd* z, const SolveBufs& B, bool add) {
  const Plan& P = c->P;
  cudaStream_t s = c->stream;
  cudaError_t e = nn_rms(v, S, P.N, B.nn_rms, s);
  c->launches++;
  const long per = (long)(P.L - 1) * P.nt;
  for (int s0 = 0; s0 < S && e == cudaSuccess; s0 += P.nn_cs) {
    const int ns = std::min(P.nn_cs, S - s0);
    const long Pn = ns * per;
    e = nn_features(v, s0, ns, P.L, P.nt, B.nn_rms, B.nn_X, Pn, s);
    if (e == cudaSuccess) e = nn_forward(c->d.nn_wbf, c->d.nn_theta, B.nn_X, Pn, P.nt, nullptr, B.nn_A, B.nn_Y, s);
    if (e == cudaSuccess) e = nn_unfeatures(B.nn_Y, s0, ns, P.L, P.nt, B.nn_rms, z, add, s);
    c->launches += 6;
  }
  return e;
}

// Training buffers for P positions: features, targets, kept pre-activations and
// activations, outputs and their gradient, two W x P gradient buffers.
struct NnBufs {
  float *X, *T, *H, *A, *Y, *dY, *dA, *dH;
};
NnBufs carve_nn(Carver& c, long P) {
  NnBufs b{};
  b.X = c.take<float>((size_t)kNnCin * P);
  b.T = c.take<float>((size_t)kNnCin * P);
  b.H = c.take<float>((size_t)3 * kNnW * P);
  b.A = c.take<float>((size_t)3 * kNnW * P);
  b.Y = c.take<float>((size_t)kNnCin * P);
  b.dY = c.take<float>((size_t)kNnCin * P);
  b.dA = c.take<float>((size_t)kNnW * P);
  b.dH = c.take<float>((size_t)kNnW * P);
  return b;
}

// Seeded default weights: uniform with variance 1 / fan-in for W1..W3 (splitmix64
// stream), zero last layer and biases, so the initial correction is zero.
void nn_default_init(std::vector<float>& th, uint64_t seed) {
  uint64_t st = seed;
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  th.assign(kNnParams, 0.f);
  auto fill = [&](size_t off, size_t n, double fan_in) {
    const double a = std::sqrt(3.0 / fan_in);
    for (size_t q = 0; q < n; ++q) th[off + q] = (float)((2.0 * ((double)(next() >> 11) * 0x1.0p-53) - 1.0) * a);
  };
  fill(kNnOffW1, (size_t)kNnW * kNnCin * kNnK1, kNnCin * kNnK1);
  fill(kNnOffW2, (size_t)kNnW * kNnW, kNnW);
  fill(kNnOffW3, (size_t)kNnW * kNnW, kNnW);
}

pt_status nn_upload(pt_ctx* c, const float* host) {
  cudaStream_t s = c->stream;
  PT_CUDA(cudaMemcpyAsync(c->d.nn_theta, host, kNnParams * sizeof(float), cudaMemcpyHostToDevice, s));
  PT_CUDA(cudaMemsetAsync(c->d.nn_m, 0, kNnParams * sizeof(float), s));
  PT_CUDA(cudaMemsetAsync(c->d.nn_v, 0, kNnParams * sizeof(float), s));
  PT_CUDA(nn_to_bf16(c->d.nn_theta, c->d.nn_wbf, s));
  PT_CUDA(cudaStreamSynchronize(s));
  c->nn_t = 0;
  c->nn_ready = true;
  return PT_OK;
}

}  // namespace

extern "C" pt_status pt_last_solve_cycles(const pt_ctx* ctx, int32_t* cycles, int32_t* learned_cycles) {
  if (!ctx) return fail(PT_ERR_ARG, "ctx is NULL");
  if (cycles) *cycles = ctx->last_cycles;
  if (learned_cycles) *learned_cycles = ctx->learned_used;
  return PT_OK;
}

extern "C" pt_status pt_last_solve_relaxed(const pt_ctx* ctx, int32_t* relaxed_matvecs) {
  if (!ctx || !relaxed_matvecs) return fail(PT_ERR_ARG, "NULL argument");
  *relaxed_matvecs = ctx->relaxed_matvecs;
  return PT_OK;
}

extern "C" pt_status pt_correction_nparams(int64_t* nparams) {
  if (!nparams) return fail(PT_ERR_ARG, "nparams is NULL");
  *nparams = (int64_t)kNnParams;
  return PT_OK;
}

extern "C" pt_status pt_set_correction(pt_ctx* ctx, const float* params, int64_t nparams) {
  if (!ctx || !params) return fail(PT_ERR_ARG, "bad arguments");
  if (nparams != (int64_t)kNnParams) return fail(PT_ERR_ARG, "nparams does not match the network");
  return nn_upload(ctx, params);
}

extern "C" pt_status pt_get_correction(const pt_ctx* ctx, float* params, int64_t nparams) {
  if (!ctx || !params) return fail(PT_ERR_ARG, "bad arguments");
  if (nparams != (int64_t)kNnParams) return fail(PT_ERR_ARG, "nparams does not match the network");
  if (!ctx->nn_ready) return fail(PT_ERR_ARG, "no correction weights set or trained");
  PT_CUDA(cudaMemcpyAsync(params, ctx->d.nn_theta, kNnParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_correction_scratch_bytes(const pt_ctx* ctx, int32_t nseq, size_t* bytes) {
  if (!ctx || !bytes || nseq < 1) return fail(PT_ERR_ARG, "bad arguments");
  Carver c(nullptr);
  carve_nn(c, (long)nseq * ctx->P.nt);
  *bytes = c.off;
  return PT_OK;
}

extern "C" pt_status pt_correction_forward(pt_ctx* ctx, int32_t nseq, const float* x, float* y, void* scratch,
                                           size_t scratch_bytes) {
  if (!ctx || !x || !y || !scratch || nseq < 1) return fail(PT_ERR_ARG, "bad arguments");
  if (!ctx->nn_ready) return fail(PT_ERR_ARG, "no correction weights set or trained");
  size_t need = 0;
  pt_correction_scratch_bytes(ctx, nseq, &need);
  if (scratch_bytes < need) return fail(PT_ERR_WORKSPACE, "scratch too small");
  Carver c(scratch);
  const long P = (long)nseq * ctx->P.nt;
  NnBufs b = carve_nn(c, P);
  PT_CUDA(nn_forward(ctx->d.nn_wbf, ctx->d.nn_theta, x, P, ctx->P.nt, nullptr, b.A, y, ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_correction_grad(pt_ctx* ctx, int32_t nseq, const float* x, const float* t, double* loss,
                                        float* grad, void* scratch, size_t scratch_bytes) {
  if (!ctx || !x || !t || !grad || !scratch || nseq < 1) return fail(PT_ERR_ARG, "bad arguments");
  if (!ctx->nn_ready) return fail(PT_ERR_ARG, "no correction weights set or trained");
  size_t need = 0;
  pt_correction_scratch_bytes(ctx, nseq, &need);
  if (scratch_bytes < need) return fail(PT_ERR_WORKSPACE, "scratch too small");
  Carver c(scratch);
  const long P = (long)nseq * ctx->P.nt;
  NnBufs b = carve_nn(c, P);
  cudaStream_t s = ctx->stream;
  PT_CUDA(cudaMemsetAsync(grad, 0, kNnParams * sizeof(float), s));
  PT_CUDA(cudaMemsetAsync(ctx->d.nn_loss, 0, sizeof(double), s));
  PT_CUDA(nn_forward(ctx->d.nn_wbf, ctx->d.nn_theta, x, P, ctx->P.nt, b.H, b.A, b.Y, s));
  PT_CUDA(nn_backward(ctx->d.nn_wbf, x, P, ctx->P.nt, b.H, b.A, b.Y, t, b.dY, b.dA, b.dH, grad, ctx->d.nn_loss, s));
  double l = 0.0;
  PT_CUDA(cudaMemcpyAsync(&l, ctx->d.nn_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  PT_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = l;
  return PT_OK;
}

namespace {
struct TrainBufs {
  void* solve;  // solve scratch (K^{-1} of the targets)
  float *Xall, *Tall;
  double* rms;
  int* idx;
  NnBufs nb;
};
TrainBufs carve_train(const pt_ctx* ctx, int npairs, int batch, void* base, size_t* bytes) {
  const Plan& P = ctx->P;
  size_t sb = 0;
  carve_solve(P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &sb);
  Carver c(base);
  TrainBufs t{};
  t.solve = c.take<unsigned char>(sb);
  const long per = (long)(P.L - 1) * P.nt;
  t.Xall = c.take<float>((size_t)kNnCin * npairs * per);
  t.Tall = c.take<float>((size_t)kNnCin * npairs * per);
  t.rms = c.take<double>(npairs);
  t.idx = c.take<int>(batch);
  t.nb = carve_nn(c, (long)batch * per);
  if (bytes) *bytes = c.off;
  return t;
}
}  // namespace

extern "C" pt_status pt_train_bytes(const pt_ctx* ctx, int32_t npairs, int32_t batch, size_t* bytes) {
  if (!ctx || !bytes || npairs < 1 || batch < 1 || batch > npairs) return fail(PT_ERR_ARG, "bad arguments");
  carve_train(ctx, npairs, batch, nullptr, bytes);
  return PT_OK;
}

extern "C" pt_status pt_train_correction(pt_ctx* ctx, int32_t npairs, const pt_c128* r, const pt_c128* e,
                                         int32_t steps, int32_t batch, double lr, uint64_t seed, double* loss_first,
                                         double* loss_last, void* scratch, size_t scratch_bytes) {
  if (!ctx || !r || !e || !scratch || npairs < 1 || batch < 1 || batch > npairs || steps < 0 || !(lr > 0))
    return fail(PT_ERR_ARG, "bad arguments");
  if ((uintptr_t)scratch % kAlign) return fail(PT_ERR_ARG, "scratch must be 256-byte aligned");
  size_t need = 0;
  carve_train(ctx, npairs, batch, nullptr, &need);
  if (scratch_bytes < need) return fail(PT_ERR_WORKSPACE, "scratch too small");
  TrainBufs tb = carve_train(ctx, npairs, batch, scratch, nullptr);
  const Plan& P = ctx->P;
  cudaStream_t s = ctx->stream;
  if (!ctx->nn_ready) {
    std::vector<float> th;
    nn_default_init(th, seed);
    pt_status st = nn_upload(ctx, th.data());
    if (st != PT_OK) return st;
  }
  // targets (e - K^{-1} r) / RMS(r) and inputs P r / RMS(r) as features, max_sources pairs at a time
  SolveBufs B = carve_solve(P, ctx->prm.max_sources, ctx->prm.max_krylov, false, tb.solve, nullptr);
  const long per = (long)(P.L - 1) * P.nt;
  const long Pall = (long)npairs * per;
  const cd* rd = reinterpret_cast<const cd*>(r);
  const cd* ed = reinterpret_cast<const cd*>(e);
  for (int p0 = 0; p0 < npairs; p0 += ctx->prm.max_sources) {
    const int ns = std::min(ctx->prm.max_sources, npairs - p0);
    {
      pt_status bs = bind_call(ctx, B, ns);
      if (bs != PT_OK) return bs;
    }
    const cd* rp = rd + (size_t)p0 * P.N;
    PT_CUDA(do_precond(ctx, ns, rp, B.x, B.t, B.u1));
    PT_CUDA(nn_sub(ed + (size_t)p0 * P.N, B.x, B.w, (size_t)ns * P.N, s));
    PT_CUDA(nn_rms(rp, ns, P.N, tb.rms + p0, s));
    PT_CUDA(nn_features(rp, 0, ns, P.L, P.nt, tb.rms + p0, tb.Xall + (size_t)p0 * per, Pall, s));
    PT_CUDA(nn_features(B.w, 0, ns, P.L, P.nt, tb.rms + p0, tb.Tall + (size_t)p0 * per, Pall, s));
  }
  // Train on targets scaled to unit RMS (tau = 1 / RMS): the last layer is linear, so
  // W4 and b4 are multiplied by tau before and divided by it after, and the
  // stored network keeps predicting the unscaled defect.  Adam restarts per call.
  double tau = 1.0;
  {
    PT_CUDA(cudaMemsetAsync(ctx->d.nn_loss + 1, 0, sizeof(double), s));
    PT_CUDA(nn_sumsq(tb.Tall, (long)kNnCin * Pall, ctx->d.nn_loss + 1, s));
    double ss = 0.0;
    PT_CUDA(cudaMemcpyAsync(&ss, ctx->d.nn_loss + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    PT_CUDA(cudaStreamSynchronize(s));
    const double rmsT = std::sqrt(ss / ((double)kNnCin * Pall));
    if (rmsT > 0.0 && std::isfinite(rmsT)) tau = 1.0 / rmsT;
  }
  PT_CUDA(nn_scale(tb.Tall, (long)kNnCin * Pall, (float)tau, s));
  PT_CUDA(nn_scale(ctx->d.nn_theta + kNnOffW4, (long)(kNnParams - kNnOffW4), (float)tau, s));
  PT_CUDA(cudaMemsetAsync(ctx->d.nn_m, 0, kNnParams * sizeof(float), s));
  PT_CUDA(cudaMemsetAsync(ctx->d.nn_v, 0, kNnParams * sizeof(float), s));
  PT_CUDA(nn_to_bf16(ctx->d.nn_theta, ctx->d.nn_wbf, s));
  ctx->nn_t = 0;
  // Adam on minibatches drawn without replacement within each pass over the pairs
  std::vector<int> order(npairs), pick(batch);
  for (int q = 0; q < npairs; ++q) order[q] = q;
  uint64_t st = seed ^ 0x5DEECE66Dull;
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto shuffle = [&]() {
    for (int q = npairs - 1; q > 0; --q) std::swap(order[q], order[next() % (uint64_t)(q + 1)]);
  };
  shuffle();
  int cursor = 0;
  const long Pb = (long)batch * per;
  for (int it = 0; it < steps; ++it) {
    for (int q = 0; q < batch; ++q) {
      if (cursor == npairs) { shuffle(); cursor = 0; }
      pick[q] = order[cursor++];
    }
    PT_CUDA(cudaMemcpyAsync(tb.idx, pick.data(), batch * sizeof(int), cudaMemcpyHostToDevice, s));
    PT_CUDA(nn_gather(tb.Xall, Pall, tb.idx, batch, P.L - 1, P.nt, tb.nb.X, s));
    PT_CUDA(nn_gather(tb.Tall, Pall, tb.idx, batch, P.L - 1, P.nt, tb.nb.T, s));
    PT_CUDA(cudaMemsetAsync(ctx->d.nn_grad, 0, kNnParams * sizeof(float), s));
    PT_CUDA(cudaMemsetAsync(ctx->d.nn_loss, 0, sizeof(double), s));
    PT_CUDA(nn_forward(ctx->d.nn_wbf, ctx->d.nn_theta, tb.nb.X, Pb, P.nt, tb.nb.H, tb.nb.A, tb.nb.Y, s));
    PT_CUDA(nn_backward(ctx->d.nn_wbf, tb.nb.X, Pb, P.nt, tb.nb.H, tb.nb.A, tb.nb.Y, tb.nb.T, tb.nb.dY, tb.nb.dA,
                        tb.nb.dH, ctx->d.nn_grad, ctx->d.nn_loss, s));
    PT_CUDA(nn_adam(ctx->d.nn_theta, ctx->d.nn_m, ctx->d.nn_v, ctx->d.nn_grad, ctx->d.nn_wbf, lr, ++ctx->nn_t, s));
    if (it == 0 || it == steps - 1) {
      double l = 0.0;
      PT_CUDA(cudaMemcpyAsync(&l, ctx->d.nn_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
      PT_CUDA(cudaStreamSynchronize(s));
      // losses are reported in the unscaled units of the defect
      if (it == 0 && loss_first) *loss_first = l / (tau * tau);
      if (it == steps - 1 && loss_last) *loss_last = l / (tau * tau);
    }
  }
  PT_CUDA(nn_scale(ctx->d.nn_theta + kNnOffW4, (long)(kNnParams - kNnOffW4), (float)(1.0 / tau), s));
  PT_CUDA(nn_to_bf16(ctx->d.nn_theta, ctx->d.nn_wbf, s));
  PT_CUDA(cudaStreamSynchronize(s));
  pt_status stt = read_status(ctx);
  return stt;
}

extern "C" pt_status pt_apply_correction(pt_ctx* ctx, int32_t nsrc, const pt_c128* v, pt_c128* z, void* scratch,
                                         size_t scratch_bytes) {
  if (!ctx || !v || !z) return fail(PT_ERR_ARG, "bad arguments");
  if (!ctx->P.learned) return fail(PT_ERR_ARG, "context created with learned = 0");
  if (!ctx->nn_ready) return fail(PT_ERR_ARG, "no correction weights set or trained");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  PT_CUDA(do_correction(ctx, nsrc, reinterpret_cast<const cd*>(v), reinterpret_cast<cd*>(z), B, false));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_plr_stats(const pt_ctx* ctx, int64_t* stored_entries, int32_t* leaves) {
  if (!ctx) return fail(PT_ERR_ARG, "ctx is NULL");
  if (stored_entries) *stored_entries = (int64_t)ctx->plr_stored;
  if (leaves) *leaves = ctx->plr_leaves;
  return PT_OK;
}

extern "C" pt_status pt_apply_R(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y) {
  if (!ctx || !x || !y || nsrc < 1 || nsrc > ctx->prm.max_sources) return fail(PT_ERR_ARG, "bad arguments");
  PT_CUDA(do_R(ctx, nsrc, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y), kModeFP64));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_apply_D_inverse(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y) {
  if (!ctx || !x || !y || x == y || nsrc < 1 || nsrc > ctx->prm.max_sources) return fail(PT_ERR_ARG, "bad arguments");
  PT_CUDA(do_Dinv(ctx, nsrc, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y), kModeFP64));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_apply_precond(pt_ctx* ctx, int32_t nsrc, const pt_c128* x, pt_c128* y, void* scratch,
                                      size_t scratch_bytes) {
  if (!ctx || !x || !y || x == y) return fail(PT_ERR_ARG, "bad arguments");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  st = bind_call(ctx, B, nsrc);
  if (st != PT_OK) return st;
  PT_CUDA(do_precond(ctx, nsrc, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y), B.t, B.u1));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_rhs(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* y, void* scratch,
                            size_t scratch_bytes) {
  if (!ctx || !f || !y) return fail(PT_ERR_ARG, "bad arguments");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  const cd* fd = reinterpret_cast<const cd*>(f);
  PT_CUDA(launch_layer_nonzero(ctx->P.g, ctx->d.layers, fd, B.nzflag, nullptr, nsrc, ctx->stream));
  PT_CUDA(launch_layer_solve(0, ctx->P.g, ctx->d.layers, ctx->d.Sinv, ctx->d.W, ctx->d.E, fd, nullptr, B.Y,
                             (size_t)ctx->P.nt * ctx->P.nloc_max, reinterpret_cast<cd*>(y), B.nzflag, nsrc,
                             ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_get_block(pt_ctx* ctx, int32_t layer, int32_t j, int32_t k, pt_c128* dst) {
  if (!ctx || !dst || layer < 0 || layer >= ctx->P.L) return fail(PT_ERR_ARG, "bad arguments");
  const LayerInfo& I = ctx->P.layers[layer];
  auto idx = [&](int q) -> int {
    if (I.has_top && q == 0) return 0;
    if (I.has_top && q == 1) return 1;
    if (I.has_bot && q == I.n) return 2;
    if (I.has_bot && q == I.n + 1) return 3;
    return -1;
  };
  int jj = idx(j), kk = idx(k);
  if (jj < 0 || kk < 0) return fail(PT_ERR_ARG, "j, k must be trace rows of the layer");
  const size_t bsz = (size_t)ctx->P.nt * ctx->P.nt;
  PT_CUDA(cudaMemcpyAsync(dst, ctx->d.blocks + ((size_t)layer * 16 + jj * 4 + kk) * bsz, bsz * sizeof(cd),
                          cudaMemcpyDeviceToDevice, ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}

extern "C" pt_status pt_last_solve_stats(const pt_ctx* ctx, int64_t* kernel_launches, int32_t* max_iterations) {
  if (!ctx) return fail(PT_ERR_ARG, "ctx is NULL");
  if (kernel_launches) *kernel_launches = ctx->launches;
  if (max_iterations) *max_iterations = ctx->last_max_it;
  return PT_OK;
}

// ---- flexible GMRES (Section 4.2) -------------------------------------------
static pt_status solve_impl(pt_ctx* c, int S, const cd* f, cd* u, cd* traces, double tol, int max_it,
                            const SolveBufs& B, int32_t* iters_out, double* relres_out) {
  const Plan& P = c->P;
  const size_t N = P.N;
  const int m = c->prm.max_krylov;
  cudaStream_t s = c->stream;
  c->launches = 0;
  {
    pt_status bs = bind_call(c, B, S);
    if (bs != PT_OK) return bs;
  }
  std::vector<double> beta(S), rel(S, 1.0);
  std::vector<int> done(S, 0), kk(S, 0), total(S, 0);
  c->resid_h.assign(S, 0.0);

  PT_CUDA(cudaMemsetAsync(c->d.status, 0, sizeof(int), s));
  PT_CUDA(do_rhs(c, S, f, B.b, B));  // P b
  PT_CUDA(cudaMemsetAsync(B.x, 0, S * N * sizeof(cd), s));
  // r = P b (x0 = 0)
  PT_CUDA(cudaMemcpyAsync(B.w, B.b, S * N * sizeof(cd), cudaMemcpyDeviceToDevice, s));
  bool first = true;
  int used = 0;
  std::vector<double> nrm(S);
  // learned correction: on while every cycle that used it at least halved the true residual
  bool learned_on = c->opt_learned && c->nn_ready && P.learned;
  std::vector<double> rel_prev(S, 1.0);
  c->learned_used = 0;
  c->last_cycles = 0;
  c->relaxed_matvecs = 0;
  while (true) {
    // V_0 = r / ||r||, g = (||r||, 0, ...), H = 0
    PT_CUDA(cudaMemsetAsync(B.H, 0, (size_t)S * (m + 1) * m * sizeof(cd), s));
    PT_CUDA(cudaMemsetAsync(B.g, 0, (size_t)S * (m + 1) * sizeof(cd), s));
    c->launches++;
    PT_CUDA(launch_norm_scale(B.w, N, S, B.nrm, B.g, 1, m + 1, 0, 0, B.V, N, reinterpret_cast<double*>(B.partial), s));
    PT_CUDA(cudaMemcpyAsync(nrm.data(), B.nrm, S * sizeof(double), cudaMemcpyDeviceToHost, s));
    PT_CUDA(cudaStreamSynchronize(s));
    if (first) {
      for (int q = 0; q < S; ++q) {
        beta[q] = nrm[q];
        if (beta[q] == 0.0) { done[q] = 1; rel[q] = 0.0; }
      }
      first = false;
    }
    std::vector<int> active(S, 0);
    int nact = 0;
    // Cycle target: tol ||P b||.  In PT_MIXED_TC the tensor-core matvec (~1e-5 relative)
    // lets the true residual stall near 1e-4 of the cycle's starting residual: a cycle
    // that cannot reach tol stops 3e-4 below its start (further iterations would be
    // lost until the double-float restart); one that can aims at 0.3 tol, so that the
    // true residual, its estimate plus that floor, lands under tol without another
    // restart.
    std::vector<double> target(S);
    for (int q = 0; q < S; ++q) {
      kk[q] = 0;
      if (!done[q]) { active[q] = 1; nact++; }
      target[q] = tol * beta[q];
      if (tcmode(c)) target[q] = 3e-4 * nrm[q] > tol * beta[q] ? 3e-4 * nrm[q] : 0.3 * tol * beta[q];
    }
    if (nact == 0 || used >= max_it) break;
    c->last_cycles++;
    int j = 0;
    for (; j < m && used < max_it; ++j) {
      cd* Vj = B.V + (size_t)j * S * N;
      cd* Zj = B.Z + (size_t)j * S * N;
      PT_CUDA(do_precond(c, S, Vj, Zj, B.t, B.u1));
      if (learned_on) PT_CUDA(do_correction(c, S, Vj, Zj, B, /*add=*/true));
      // Inexact Krylov relaxation (mixed FP32 form): once every active source's residual estimate
      // is below kRelax tol ||b||, the matvec's error may grow as tol ||b|| / ||r||, and the FP32
      // product (~1e-6 relative) replaces the double-float one; the residual gap it opens is at
      // most about 2e-6 ||r|| per relaxed step, below 1e-2 tol ||b|| in all, and the restart
      // residual stays double-float
      bool relax = c->opt_relax && c->prm.precision == PT_MIXED_FP32 && !c->P.plr && j > 0;
      for (int q = 0; q < S && relax; ++q)
        if (active[q] && !kk[q] && !(c->resid_h[q] <= kRelax * tol * beta[q])) relax = false;
      if (relax) {
        c->relaxed_matvecs++;
        PT_CUDA(apply(c, kModeFP32, op_matvec(c), S, Zj, nullptr, B.w, kApplyRowsWide, 1.0, 0.0, true));
      } else {
        PT_CUDA(do_matvec(c, S, Zj, B.w, /*exact=*/false));
      }
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        c->launches += 3;
        PT_CUDA(launch_dots(B.V, S, N, B.w, j + 1, B.partial, B.coef, m + 1, B.H, m + 1, m, j, s));
        PT_CUDA(launch_update(B.V, S, N, B.w, j + 1, B.coef, m + 1, s));
      }
      c->launches += 2;
      PT_CUDA(launch_norm_scale(B.w, N, S, nullptr, B.H, m + 1, m, j + 1, j, B.V + (size_t)(j + 1) * S * N, N,
                                reinterpret_cast<double*>(B.partial), s));
      PT_CUDA(launch_givens(S, m, j, B.H, B.cs, B.sn, B.g, B.resid, s));
      PT_CUDA(cudaMemcpyAsync(c->resid_h.data(), B.resid, S * sizeof(double), cudaMemcpyDeviceToHost, s));
      PT_CUDA(cudaStreamSynchronize(s));
      used++;
      bool all = true;
      for (int q = 0; q < S; ++q) {
        if (!active[q] || kk[q]) continue;
        if (!(c->resid_h[q] > target[q])) kk[q] = j + 1;  // cycle done (or NaN: stop it too)
        else all = false;
      }
      if (all) { ++j; break; }
    }
    for (int q = 0; q < S; ++q) {
      if (active[q] && !kk[q]) kk[q] = j;
      total[q] += active[q] ? kk[q] : 0;
    }
    PT_CUDA(cudaMemcpyAsync(B.kk, kk.data(), S * sizeof(int), cudaMemcpyHostToDevice, s));
    c->launches += 2;
    PT_CUDA(launch_lsq_combine(S, m, B.kk, B.H, B.g, B.y, B.Z, N, B.x, s));
    // explicit residual r = P b - P M x between restart cycles (iterative refinement)
    PT_CUDA(do_restart_matvec(c, S, B.x, B.t));
    c->launches += 2;
    PT_CUDA(launch_sub(B.b, B.t, B.w, S * N, s));
    PT_CUDA(launch_norm_scale(B.w, N, S, B.nrm, nullptr, 0, 0, 0, 0, nullptr, 0, reinterpret_cast<double*>(B.partial),
                              s));
    PT_CUDA(cudaMemcpyAsync(nrm.data(), B.nrm, S * sizeof(double), cudaMemcpyDeviceToHost, s));
    PT_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    bool poor = false;
    for (int q = 0; q < S; ++q) {
      if (done[q]) continue;
      rel[q] = nrm[q] / beta[q];
      if (!(rel[q] <= 0.5 * rel_prev[q])) poor = true;
      rel_prev[q] = rel[q];
      if (rel[q] <= tol) done[q] = 1;
      else all = false;
    }
    if (learned_on) {
      c->learned_used++;
      if (poor) learned_on = false;  // fall back to the plain preconditioner
    }
    if (all || used >= max_it) break;
  }
  // outputs
  if (traces) PT_CUDA(cudaMemcpyAsync(traces, B.x, S * N * sizeof(cd), cudaMemcpyDeviceToDevice, s));
  if (u) PT_CUDA(do_layer_solve(c, 1, S, f, B.x, u, B));
  PT_CUDA(cudaStreamSynchronize(s));
  pt_status st = read_status(c);
  if (st != PT_OK) return st;
  int maxit = 0;
  bool conv = true;
  for (int q = 0; q < S; ++q) {
    if (iters_out) iters_out[q] = total[q];
    if (relres_out) relres_out[q] = rel[q];
    maxit = std::max(maxit, total[q]);
    if (!(rel[q] <= tol)) conv = false;
  }
  c->last_max_it = maxit;
  if (!conv) return fail(PT_ERR_NOT_CONVERGED, "GMRES reached max_it before rel_tol");
  return PT_OK;
}

extern "C" pt_status pt_solve(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* u, pt_c128* traces,
                              double rel_tol, int32_t max_it, void* scratch, size_t scratch_bytes, int32_t* iters,
                              double* relres) {
  if (!ctx || !f) return fail(PT_ERR_ARG, "ctx or f is NULL");
  if (!(rel_tol > 0) || max_it < 1) return fail(PT_ERR_ARG, "rel_tol > 0 and max_it >= 1 required");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  return solve_impl(ctx, nsrc, reinterpret_cast<const cd*>(f), reinterpret_cast<cd*>(u),
                    reinterpret_cast<cd*>(traces), rel_tol, max_it, B, iters, relres);
}

// ---- Gauss-Seidel iteration as a solver (Algorithm 3, Section 4.1) -----------
// u^0 = 0; u^{k+1} = D^{-1}(P b - R u^k) while ||u^{k+1} - u^k|| / ||u^k|| > tol, with the
// exact FP64 operators in every precision form (the iteration converges to the accuracy of
// the operators it applies); then the FP64 true residual and the reconstruction of pt_solve.
static pt_status solve_gs_impl(pt_ctx* c, int S, const cd* f, cd* u, cd* traces, double tol, int max_it,
                               const SolveBufs& B, int32_t* iters_out, double* relres_out) {
  const size_t N = c->P.N;
  cudaStream_t s = c->stream;
  c->launches = 0;
  {
    pt_status bs = bind_call(c, B, S);
    if (bs != PT_OK) return bs;
  }
  std::vector<double> nrm_old(S, 0.0), nrm_new(S), nrm_diff(S);
  std::vector<int> done(S, 0), its(S, 0);
  PT_CUDA(cudaMemsetAsync(c->d.status, 0, sizeof(int), s));
  PT_CUDA(do_rhs(c, S, f, B.b, B));  // P b
  PT_CUDA(cudaMemsetAsync(B.x, 0, S * N * sizeof(cd), s));
  double* partial = reinterpret_cast<double*>(B.partial);
  for (int k = 1; k <= max_it; ++k) {
    PT_CUDA(do_R(c, S, B.x, B.t, kModeFP64, -1.0, 1.0, B.b, false));  // t = P b - R u^k
    PT_CUDA(do_Dinv(c, S, B.t, B.u1, kModeFP64, false));              // u^{k+1} = D^{-1} t
    c->launches += 3;
    PT_CUDA(launch_sub(B.u1, B.x, B.w, S * N, s));
    PT_CUDA(launch_norm_scale(B.w, N, S, B.nrm, nullptr, 0, 0, 0, 0, nullptr, 0, partial, s));
    PT_CUDA(cudaMemcpyAsync(nrm_diff.data(), B.nrm, S * sizeof(double), cudaMemcpyDeviceToHost, s));
    PT_CUDA(launch_norm_scale(B.u1, N, S, B.nrm, nullptr, 0, 0, 0, 0, nullptr, 0, partial, s));
    PT_CUDA(cudaMemcpyAsync(nrm_new.data(), B.nrm, S * sizeof(double), cudaMemcpyDeviceToHost, s));
    // sources that have converged keep their iterate: copy only the active ones
    for (int q = 0; q < S; ++q)
      if (!done[q])
        PT_CUDA(cudaMemcpyAsync(B.x + (size_t)q * N, B.u1 + (size_t)q * N, N * sizeof(cd), cudaMemcpyDeviceToDevice,
                                s));
    PT_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int q = 0; q < S; ++q) {
      if (done[q]) continue;
      its[q] = k;
      const bool zero = nrm_new[q] == 0.0 && nrm_diff[q] == 0.0;  // a zero source: u = 0 is exact
      if (zero || (nrm_old[q] > 0.0 && nrm_diff[q] <= tol * nrm_old[q])) done[q] = 1;
      else all = false;
      nrm_old[q] = nrm_new[q];
    }
    if (all) break;
  }
  // FP64 true residual ||P b - P M u|| / ||P b||
  PT_CUDA(do_matvec(c, S, B.x, B.t));
  c->launches += 3;
  PT_CUDA(launch_sub(B.b, B.t, B.w, S * N, s));
  std::vector<double> rn(S), bn(S);
  PT_CUDA(launch_norm_scale(B.w, N, S, B.nrm, nullptr, 0, 0, 0, 0, nullptr, 0, partial, s));
  PT_CUDA(cudaMemcpyAsync(rn.data(), B.nrm, S * sizeof(double), cudaMemcpyDeviceToHost, s));
  PT_CUDA(launch_norm_scale(B.b, N, S, B.nrm, nullptr, 0, 0, 0, 0, nullptr, 0, partial, s));
  PT_CUDA(cudaMemcpyAsync(bn.data(), B.nrm, S * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (traces) PT_CUDA(cudaMemcpyAsync(traces, B.x, S * N * sizeof(cd), cudaMemcpyDeviceToDevice, s));
  if (u) PT_CUDA(do_layer_solve(c, 1, S, f, B.x, u, B));
  PT_CUDA(cudaStreamSynchronize(s));
  pt_status st = read_status(c);
  if (st != PT_OK) return st;
  bool conv = true;
  int maxit = 0;
  for (int q = 0; q < S; ++q) {
    if (iters_out) iters_out[q] = its[q];
    if (relres_out) relres_out[q] = bn[q] > 0.0 ? rn[q] / bn[q] : 0.0;
    maxit = std::max(maxit, its[q]);
    if (!done[q]) conv = false;
  }
  c->last_max_it = maxit;
  if (!conv) return fail(PT_ERR_NOT_CONVERGED, "Gauss-Seidel reached max_it before rel_tol");
  return PT_OK;
}

extern "C" pt_status pt_solve_gs(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* u, pt_c128* traces,
                                 double rel_tol, int32_t max_it, void* scratch, size_t scratch_bytes, int32_t* iters,
                                 double* relres) {
  if (!ctx || !f) return fail(PT_ERR_ARG, "ctx or f is NULL");
  if (!(rel_tol > 0) || max_it < 1) return fail(PT_ERR_ARG, "rel_tol > 0 and max_it >= 1 required");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, false, scratch, nullptr);
  return solve_gs_impl(ctx, nsrc, reinterpret_cast<const cd*>(f), reinterpret_cast<cd*>(u),
                       reinterpret_cast<cd*>(traces), rel_tol, max_it, B, iters, relres);
}

extern "C" pt_status pt_solve_many(int32_t nctx, pt_ctx* const* ctxs, const int32_t* nsrc, const pt_c128* const* f,
                                   pt_c128* const* u, double rel_tol, int32_t max_it, void* const* scratch,
                                   const size_t* scratch_bytes, int32_t* iters, double* relres, int32_t* status) {
  if (nctx < 1 || !ctxs || !nsrc || !f || !scratch || !scratch_bytes) return fail(PT_ERR_ARG, "bad arguments");
  std::vector<size_t> off(nctx + 1, 0);
  for (int k = 0; k < nctx; ++k) {
    if (!ctxs[k]) return fail(PT_ERR_ARG, "a context is NULL");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(PT_ERR_ARG, "a context appears twice");
    if (nsrc[k] < 1) return fail(PT_ERR_ARG, "nsrc must be >= 1");
    off[k + 1] = off[k] + (size_t)nsrc[k];
  }
  int dev = 0;
  PT_CUDA(cudaGetDevice(&dev));
  std::vector<pt_status> st(nctx, PT_OK);
  std::vector<std::string> msg(nctx);
  auto work = [&](int k) {
    g_shared_gpu = true;
    if (cudaSetDevice(dev) != cudaSuccess) {
      st[k] = PT_ERR_CUDA;
      msg[k] = "cudaSetDevice failed";
      return;
    }
    st[k] = pt_solve(ctxs[k], nsrc[k], f[k], u ? u[k] : nullptr, nullptr, rel_tol, max_it, scratch[k],
                     scratch_bytes[k], iters ? iters + off[k] : nullptr, relres ? relres + off[k] : nullptr);
    if (st[k] != PT_OK) msg[k] = pt_last_error();
  };
  std::vector<std::thread> pool;
  pool.reserve(nctx);
  for (int k = 0; k < nctx; ++k) pool.emplace_back(work, k);
  for (auto& t : pool) t.join();
  if (status)
    for (int k = 0; k < nctx; ++k) status[k] = (int32_t)st[k];
  for (int k = 0; k < nctx; ++k)
    if (st[k] != PT_OK) return fail(st[k], ("context " + std::to_string(k) + ": " + msg[k]).c_str());
  return PT_OK;
}

extern "C" pt_status pt_solve_host(pt_ctx* ctx, int32_t nsrc, const pt_c128* f_host, pt_c128* u_host,
                                   double rel_tol, int32_t max_it, void* scratch, size_t scratch_bytes,
                                   int32_t* iters, double* relres) {
  if (!ctx || !f_host || !u_host) return fail(PT_ERR_ARG, "NULL pointer");
  if (!(rel_tol > 0) || max_it < 1) return fail(PT_ERR_ARG, "rel_tol > 0 and max_it >= 1 required");
  size_t need = 0;
  carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, true, nullptr, &need);
  pt_status st = check_solve_args(ctx, nsrc, scratch, scratch_bytes, need);
  if (st != PT_OK) return st;
  SolveBufs B = carve_solve(ctx->P, ctx->prm.max_sources, ctx->prm.max_krylov, true, scratch, nullptr);
  const size_t vol = (size_t)nsrc * ctx->P.Nz * ctx->P.nt * sizeof(cd);
  PT_CUDA(cudaMemcpyAsync(B.fdev, f_host, vol, cudaMemcpyHostToDevice, ctx->stream));
  st = solve_impl(ctx, nsrc, B.fdev, B.udev, nullptr, rel_tol, max_it, B, iters, relres);
  if (st != PT_OK && st != PT_ERR_NOT_CONVERGED) return st;
  PT_CUDA(cudaMemcpyAsync(u_host, B.udev, vol, cudaMemcpyDeviceToHost, ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return st;
}

// ---- pt_rhs_noalloc: pt_rhs without caller-provided scratch -----------------
// The local-solve storage of pt_rhs, for callers that cannot allocate device
// memory, lives in this file-scope device array.  Host code must not use the
// name g_rhs_noalloc_scratch as an address (on the host it only stands for
// the symbol); its device address is looked up once per device below.
namespace {
constexpr size_t kRhsNoallocBytes = 16u << 20;  // 16 MiB
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_rhs_noalloc_scratch[kRhsNoallocBytes];

// Device address of the array on the current device; the first call on a
// device performs the lookup (cudaGetSymbolAddress) with that device current.
static pt_status rhs_noalloc_scratch(const pt_ctx* ctx, void** out) {
  int dev = -1;
  PT_CUDA(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return fail(PT_ERR_ARG, "pt_rhs_noalloc: the current device is not the device the context was created on");
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(PT_ERR_ARG, "pt_rhs_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(PT_ERR_CUDA, std::string("pt_rhs_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return PT_OK;
}

extern "C" pt_status pt_rhs_noalloc(pt_ctx* ctx, int32_t nsrc, const pt_c128* f, pt_c128* y) {
  if (!ctx || !f || !y) return fail(PT_ERR_ARG, "pt_rhs_noalloc: NULL argument");
  if (nsrc < 1) return fail(PT_ERR_ARG, "pt_rhs_noalloc: nsrc must be >= 1");
  const Plan& P = ctx->P;
  const size_t ystride = (size_t)P.nt * P.nloc_max;
  const size_t ybytes = ((size_t)nsrc * P.L * ystride * sizeof(cd) + kAlign - 1) / kAlign * kAlign;
  const size_t need = ybytes + (size_t)nsrc * P.L * sizeof(int);
  if (need > kRhsNoallocBytes)
    return fail(PT_ERR_WORKSPACE, "pt_rhs_noalloc: needs " + std::to_string(need) +
                                      " bytes, more than its 16 MiB built-in scratch; use pt_rhs");
  void* base = nullptr;
  pt_status st = rhs_noalloc_scratch(ctx, &base);
  if (st != PT_OK) return st;
  cd* Y = static_cast<cd*>(base);
  int* flag = reinterpret_cast<int*>(static_cast<char*>(base) + ybytes);
  const cd* fd = reinterpret_cast<const cd*>(f);
  PT_CUDA(launch_layer_nonzero(P.g, ctx->d.layers, fd, flag, nullptr, nsrc, ctx->stream));
  PT_CUDA(launch_layer_solve(0, P.g, ctx->d.layers, ctx->d.Sinv, ctx->d.W, ctx->d.E, fd, nullptr, Y, ystride,
                             reinterpret_cast<cd*>(y), flag, nsrc, ctx->stream));
  PT_CUDA(cudaStreamSynchronize(ctx->stream));
  return PT_OK;
}
