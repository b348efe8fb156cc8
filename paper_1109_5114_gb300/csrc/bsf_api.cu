// C ABI of libbsf.so (declared in include/bsf.h): contexts, workspace,
// argument checking, the order of the kernel launches, and the status word.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <new>

#include "bsf_internal.h"

struct bsf_ctx {
  int H = 0, W = 0, N = 4, n = 1, boundary = BSF_SYMMETRIC;
  int R = -1;               // padding; -1 until known
  bool R_fixed = false;     // given at create
  int precision = BSF_FIX64;       // element type of the running sums in use
  bool prec_auto = false;          // BSF_FIX: the width is chosen per pre-integration
  int frac_req = -1;        // requested q (-1 = automatic)
  int q = -1;               // q of the current pre-integration
  int step_rule = BSF_STEP_D1;
  int dirset = BSF_DIRS_CARTESIAN;  // direction set (BSF_OPT_DIRECTIONS)
  int tiles = 1;                    // BSF_OPT_TILES
  int max_smem = 0;                 // opt-in shared memory per block (bytes)
  bool has_bound = false;
  double value_bound = 0.0;
  cudaStream_t stream = nullptr;
  int device = 0;

  int Hp = 0, Wp = 0;
  long long pitch = 0;
  int elem = 8;
  void* S = nullptr;
  void* S2 = nullptr;               // BSF_DIRS_PAIR: running sums of the second set
  size_t S_bytes = 0;
  void* agg = nullptr;
  void* carry = nullptr;
  size_t scan_bytes = 0;
  void* G = nullptr;               // backward: adjoint running sums [Hp][pitch] (uint64 or uint128)
  void* Gx = nullptr;              // backward: row-folded [Hp][W]
  void* bagg = nullptr;            // backward: chunk states of the reversed vertical sums
  size_t G_bytes = 0, Gx_bytes = 0, bagg_bytes = 0;
  unsigned* sync_words = nullptr;  // look-back ticket + tile flags
  size_t sync_bytes = 0;
  int scan_mode = BSF_SCAN_THREE_PHASE;
  int scan_chunk = kScanChunk;   // rows per chunk, three-phase scan
  int short_tiles = 0;           // look-back tiles of half height
  int wait_limit = 1 << 20;
  int test_unpublished = 0;
  bool plan_union = false;       // plans widen R and the mass bound instead of replacing them
  ushort4* Lf = nullptr;
  DevStatus* st = nullptr;
  DevStatus host_st{};

  bool planned = false;      // a step solve has set R and the mass bound
  double plan_mass = 1.0;    // largest prod L^n of the plan
  int plan_reach = -1;       // largest tap reach of the plan
  const float* last_cov = nullptr;  // covariance of the last filter call (bsf_copy_steps)
  int last_kind = BSF_COV_C;
  bool steps_current = false;       // Lf holds the steps of last_cov
  bool have_S = false;       // S holds a pre-integration made with (R, elem, q)
  int S_R = -1, S_elem = 0, S_q = -1, S_dirset = BSF_DIRS_CARTESIAN;
  int S_row0 = 0, S_rows = 0;        // image rows the held running sums cover
  char msg[512] = "ok";

  // host-buffer entry (bsf_filter_host): device staging copies of the inputs
  // and the output, one stream per copy direction, and the band events
  static constexpr int kHostBands = 32;  // most bands of bsf_filter_host
  int host_bands = 8;
  void* hs_img = nullptr;
  void* hs_cov = nullptr;
  void* hs_out = nullptr;
  size_t hs_img_bytes = 0, hs_cov_bytes = 0, hs_out_bytes = 0;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  cudaEvent_t hev[2 * kHostBands + 4] = {};
  bool hev_ready = false;
  // the whole host-buffer call as a CUDA graph, replayed while its key holds
  cudaStream_t s_cap = nullptr;
  cudaGraphExec_t hgraph = nullptr;
  long long hkey[18] = {};

  // Algorithm 1 (bsf_filter_two_pass): the two fields, the first pass's
  // output and the minimum of the condition-2 bound
  float* tp_fields = nullptr;  // [2][3][H][W]: isotropic, residual
  float* tp_g = nullptr;       // [H][W]
  unsigned long long* tp_min = nullptr;

  // phase timing (bsf_set_profiling)
  static constexpr int kMaxRec = 4096;
  bool profiling = false;
  cudaEvent_t* ev = nullptr;   // 2 * kMaxRec events
  int rec_phase[kMaxRec];
  int nrec = 0;
  int dropped = 0;
};

namespace {

int fail(bsf_t h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(bsf_t h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? BSF_ENOMEM : BSF_ECUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

#define BSF_CUDA(h, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

size_t elem_bytes_of(int precision) {
  return precision == BSF_FIX128 ? 16 : (precision == BSF_FIX32 ? 4 : 8);
}
bool is_fixed(int precision) {
  return precision == BSF_FIX32 || precision == BSF_FIX64 || precision == BSF_FIX128;
}
int elem_bits(int precision) { return precision == BSF_FIX128 ? 128 : (precision == BSF_FIX32 ? 32 : 64); }

void free_workspace(bsf_t h) {
  if (h->S) cudaFree(h->S);
  if (h->S2) cudaFree(h->S2);
  h->S2 = nullptr;
  if (h->agg) cudaFree(h->agg);
  if (h->carry) cudaFree(h->carry);
  if (h->sync_words) cudaFree(h->sync_words);
  if (h->G) cudaFree(h->G);
  if (h->Gx) cudaFree(h->Gx);
  if (h->bagg) cudaFree(h->bagg);
  h->G = h->Gx = h->bagg = nullptr;
  h->G_bytes = h->Gx_bytes = h->bagg_bytes = 0;
  h->S = h->agg = h->carry = nullptr;
  h->sync_words = nullptr;
  h->sync_bytes = 0;
  h->S_bytes = h->scan_bytes = 0;
  h->have_S = false;
}

// (Re)allocate S and the scan carries for the current R and precision.
int ensure_workspace(bsf_t h) {
  const int elem = (int)elem_bytes_of(h->precision);
  const int Hp = h->H + 2 * h->R, Wp = h->W + 2 * h->R;
  const long long align = 256 / elem;  // 256-byte aligned rows
  const long long pitch = (Wp + align - 1) / align * align;
  const size_t S_bytes = (size_t)pitch * Hp * elem;
  if ((long long)pitch * Hp >= (1LL << 31))
    return fail(h, BSF_EINVAL, "padded domain of %lld elements exceeds 2^31", (long long)pitch * Hp);
  const int nchunks = (Hp + kScanChunkMin - 1) / kScanChunkMin;
  size_t sync_bytes = 0;
  size_t scan_bytes = (size_t)nchunks * h->n * (size_t)(Wp + Hp - 1) * elem;
  const size_t lb_bytes = bsf_vscan_lb_bytes(elem, h->n, Hp, Wp, &sync_bytes);
  if (lb_bytes > scan_bytes) scan_bytes = lb_bytes;
  if (h->dirset != BSF_DIRS_CARTESIAN) {  // the second set's skew-2 and row-parity scans
    const size_t second = bsf_second_scan_elems(h->n, Hp, Wp, kScanChunkMin) * elem;
    if (second > scan_bytes) scan_bytes = second;
  }
  const bool need_S2 = h->dirset == BSF_DIRS_PAIR;
  if (h->S && h->S_bytes == S_bytes && h->scan_bytes >= scan_bytes && h->Hp == Hp &&
      h->Wp == Wp && h->elem == elem && (!need_S2 || h->S2))
    return BSF_OK;
  BSF_CUDA(h, cudaStreamSynchronize(h->stream));
  free_workspace(h);
  BSF_CUDA(h, cudaMalloc(&h->S, S_bytes));
  if (need_S2) BSF_CUDA(h, cudaMalloc(&h->S2, S_bytes));
  BSF_CUDA(h, cudaMalloc(&h->agg, scan_bytes));
  BSF_CUDA(h, cudaMalloc(&h->carry, scan_bytes));
  BSF_CUDA(h, cudaMalloc(&h->sync_words, sync_bytes));
  h->sync_bytes = sync_bytes;
  h->S_bytes = S_bytes;
  h->scan_bytes = scan_bytes;
  h->Hp = Hp;
  h->Wp = Wp;
  h->pitch = pitch;
  h->elem = elem;
  return BSF_OK;
}

int read_status(bsf_t h) {
  BSF_CUDA(h, cudaMemcpyAsync(&h->host_st, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
  BSF_CUDA(h, cudaStreamSynchronize(h->stream));
  return BSF_OK;
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}

double bits_to_float(unsigned b) {
  float f;
  std::memcpy(&f, &b, sizeof f);
  return (double)f;
}

// Per-call counters and maxima start from zero; the first error code is kept
// until bsf_status() reads it.
int reset_counters(bsf_t h, bool steps, bool values) {
  if (steps) {  // clamp/bad/range/overflow counts, max_reach, max_mass (0.0 bits)
    const size_t a = offsetof(DevStatus, clamp_count);
    const size_t b = offsetof(DevStatus, max_mass_bits) + sizeof(unsigned long long);
    BSF_CUDA(h, cudaMemsetAsync(reinterpret_cast<char*>(h->st) + a, 0, b - a, h->stream));
  }
  if (values) {  // max |Q|
    BSF_CUDA(h, cudaMemsetAsync(&h->st->max_absq_bits, 0, sizeof(unsigned long long), h->stream));
  }
  return BSF_OK;
}

// Scoped CUDA-event bracket of one phase execution on the context's stream.
struct PhaseTimer {
  bsf_t h;
  int slot = -1;
  PhaseTimer(bsf_t h_, int phase) : h(h_) {
    if (!h->profiling) return;
    if (h->nrec >= bsf_ctx::kMaxRec) { ++h->dropped; return; }
    slot = h->nrec++;
    h->rec_phase[slot] = phase;
    cudaEventRecord(h->ev[2 * slot], h->stream);
  }
  ~PhaseTimer() {
    if (slot >= 0) cudaEventRecord(h->ev[2 * slot + 1], h->stream);
  }
};

int check_cov_kind(bsf_t h, int cov_kind) {
  if (cov_kind != BSF_COV_C && cov_kind != BSF_COV_LOGSIG_THETA_LOGRHO)
    return fail(h, BSF_EINVAL, "unsupported cov_kind %d", cov_kind);
  return BSF_OK;
}

// Smallest padding of the sampled box spline's taps (lambda = 1 on every
// direction).
constexpr int kSampledMinPad = 4;
constexpr int kSampledMinPadSecond = 10;  // the second set's, lambda = (1, 1, 1, 1)

// Smallest padding of the continuous-step taps (identity steps): samples at
// -3..1 (n = 2) or -2..1 (n = 1) along every direction.
int d2_min_reach(int n) { return n == 2 ? 9 : 6; }

int check_d2(bsf_t h) {
  if (h->n > 2) return fail(h, BSF_EINVAL, "continuous steps need n <= 2");
  if (!is_fixed(h->precision)) return fail(h, BSF_EINVAL, "continuous steps need fixed point");
  if (h->precision == BSF_FIX32) {
    if (!h->prec_auto) return fail(h, BSF_EINVAL, "continuous steps need 64 or 128 bits");
    h->precision = BSF_FIX64;  // BSF_FIX: chosen again at the pre-integration, 64 bits at least
    h->have_S = false;
  }
  if (h->R >= 0 && h->R < d2_min_reach(h->n))
    return fail(h, BSF_EINVAL, "padding R = %d below %d, the reach of continuous identity steps",
                h->R, d2_min_reach(h->n));
  return BSF_OK;
}

// Step solve over the field; sets R and the mass bound (with a sync) when R is
// not yet known.
int run_steps(bsf_t h, const float* cov, int cov_kind, bool sync_plan) {
  int rc = check_cov_kind(h, cov_kind);
  if (rc) return rc;
  if (!cov) return fail(h, BSF_EINVAL, "cov is NULL");
  if ((rc = reset_counters(h, true, false))) return rc;
  // a plan of a context without a fixed R solves unbounded and resizes R
  const bool bounded = h->R_fixed || (h->planned && !sync_plan);
  cudaError_t e;
  {
    PhaseTimer t(h, BSF_PHASE_STEPS);
    e = bsf_launch_steps(cov, cov_kind, h->H, h->W, h->n, h->step_rule, h->dirset, bounded ? h->R : -1,
                         h->Lf, h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "steps kernel");
  h->last_cov = cov;
  h->last_kind = cov_kind;
  h->steps_current = true;
  if (sync_plan) {
    if ((rc = read_status(h))) return rc;
    const bool widen = h->plan_union && h->planned;
    const double mass = bits_to_float(h->host_st.max_mass_bits);
    const int reach = h->host_st.max_reach;
    h->plan_mass = widen && h->plan_mass > mass ? h->plan_mass : mass;
    h->plan_reach = widen && h->plan_reach > reach ? h->plan_reach : reach;
    if (!h->R_fixed) {
      // the solve ran unbounded: every tap of this field fits this R
      int R = reach > 3 * h->n ? reach : 3 * h->n;
      if (h->step_rule == BSF_STEP_D2 && R < d2_min_reach(h->n)) R = d2_min_reach(h->n);
      if (h->step_rule == BSF_STEP_SAMPLED) {
        const int minpad = h->dirset == BSF_DIRS_CARTESIAN ? kSampledMinPad : kSampledMinPadSecond;
        if (R < minpad) R = minpad;
      }
      h->R = widen && h->R > R ? h->R : R;
    }
    h->planned = true;
    if ((rc = ensure_workspace(h))) return rc;
  }
  return BSF_OK;
}

// Choose q for this pre-integration.
int resolve_q(bsf_t h, const void* img, int dtype, long long ld) {
  if (!is_fixed(h->precision)) {  // floating-point sums hold the values themselves
    h->q = 0;
    return BSF_OK;
  }
  if (h->frac_req >= 0 && !h->prec_auto) {
    h->q = h->frac_req;
    return BSF_OK;
  }
  double vmax;
  if (dtype == BSF_U8) {
    vmax = 255.0;
  } else if (h->has_bound) {
    vmax = h->value_bound;
  } else {
    BSF_CUDA(h, cudaMemsetAsync(&h->st->max_absf_bits, 0, sizeof(unsigned long long), h->stream));
    cudaError_t e = bsf_launch_absmax(img, dtype, ld, h->H, h->W, h->st, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "absmax kernel");
    int rc = read_status(h);
    if (rc) return rc;
    vmax = bits_to_double(h->host_st.max_absf_bits);
    if (!(vmax == vmax)) return fail(h, BSF_EINVAL, "image contains NaN");
  }
  // largest q with (vmax 2^q + 1/2) * mass < 2^(b-2)
  if (!h->planned)
    return fail(h, BSF_ESTATE, "automatic q needs the mass bound of a plan (bsf_plan) or explicit frac_bits");
  const double mass = h->plan_mass > 1.0 ? h->plan_mass : 1.0;
  const double lv = std::log2(vmax > 1e-300 ? vmax : 1e-300);
  const double lm = std::log2(mass);
  auto auto_q = [&](int b) {
    int q = (int)std::floor((b - 2) - lv - lm) - 1;
    if (h->step_rule == BSF_STEP_D2) q -= 2;  // derivative sums reach 3 max|Q| mass
    const int qcap = b == 32 ? 30 : b - 28;
    if (q > qcap) q = qcap;
    return q;
  };
  if (h->prec_auto) {
    // the narrowest element that holds the bound (BSF_FIX)
    static const int widths[3] = {BSF_FIX32, BSF_FIX64, BSF_FIX128};
    const int qt = dtype == BSF_U8 ? 0 : 25 - (int)std::ceil(lv);
    int pick = BSF_FIX128;
    for (int w : widths) {
      if (w == BSF_FIX32 && (h->step_rule == BSF_STEP_D2 || h->step_rule == BSF_STEP_SAMPLED))
        continue;  // continuous steps: 64 / 128 bits
      const int b = elem_bits(w);
      const bool fits = h->frac_req >= 0
                            ? std::log2((vmax * std::ldexp(1.0, h->frac_req) + 0.5) * mass) < b - 2
                            : auto_q(b) >= (qt > 0 ? qt : 0);
      if (fits) { pick = w; break; }
    }
    if (pick != h->precision) h->have_S = false;
    h->precision = pick;
    if (h->frac_req >= 0) {
      h->q = h->frac_req;
      return BSF_OK;
    }
  }
  int q = auto_q(elem_bits(h->precision));
  if (q < 0) q = 0;
  h->q = q;
  return BSF_OK;
}

// Running sums of the band of image rows [row0, row0 + rows) (the whole
// image: row0 = 0, rows = H) on its padded domain of rows + 2R rows.
int preintegrate_impl(bsf_t h, const void* img, int dtype, long long ld, int row0, int rows) {
  if (!img) return fail(h, BSF_EINVAL, "img is NULL");
  if (dtype != BSF_U8 && dtype != BSF_F32 && dtype != BSF_F64)
    return fail(h, BSF_EINVAL, "bad image dtype %d", dtype);
  if (ld < h->W) return fail(h, BSF_EINVAL, "ld %lld < W %d", ld, h->W);
  if (h->R < 0) return fail(h, BSF_ESTATE, "padding unknown: give max_reach or call bsf_plan");
  if (h->dirset != BSF_DIRS_CARTESIAN && !is_fixed(h->precision))
    return fail(h, BSF_EINVAL, "the second direction set needs fixed point");
  int rc;
  if ((rc = resolve_q(h, img, dtype, ld))) return rc;  // may choose the element (BSF_FIX)
  if ((rc = ensure_workspace(h))) return rc;
  if ((rc = reset_counters(h, false, true))) return rc;
  const int Hb = rows + 2 * h->R;  // padded rows of the band
  cudaError_t e;
  if (h->dirset != BSF_DIRS_CARTESIAN) {
    // extension + quantisation, then the running sums along e1..e4
    void* S2 = h->dirset == BSF_DIRS_PAIR ? h->S2 : h->S;
    PhaseTimer t(h, BSF_PHASE_SECOND);
    e = bsf_launch_extend(h->precision, img, dtype, ld, h->H, h->W, h->R, row0, h->boundary, h->q, S2,
                          h->pitch, Hb, h->Wp, h->st, h->stream);
    if (e == cudaSuccess)
      e = bsf_launch_scans_second(h->precision, h->n, S2, h->pitch, Hb, h->Wp, h->scan_chunk, h->agg,
                                  h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "second-set running sums");
  }
  if (h->dirset == BSF_DIRS_SECOND) {
    h->have_S = true;
    h->S_R = h->R;
    h->S_elem = h->elem;
    h->S_q = h->q;
    h->S_row0 = row0;
    h->S_rows = rows;
    h->S_dirset = h->dirset;
    return BSF_OK;
  }
  {
    PhaseTimer t(h, BSF_PHASE_ROWS);
    e = bsf_launch_scan_rows(h->precision, h->n, img, dtype, ld, h->H, h->W, h->R, row0,
                             h->boundary, h->q, h->S, h->pitch, Hb, h->Wp, h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "row scan");
  // d3, d2, d4
  const int skews[3] = {0, 1, -1};
  const int phases[3] = {BSF_PHASE_D3, BSF_PHASE_D2, BSF_PHASE_D4};
  for (int i = 0; i < 3; ++i) {
    PhaseTimer t(h, phases[i]);
    if (h->scan_mode == BSF_SCAN_LOOKBACK && is_fixed(h->precision) && h->precision != BSF_FIX32)
      e = bsf_launch_vscan_lb(h->precision, h->n, skews[i], false, h->short_tiles != 0, h->S, h->pitch,
                              Hb, h->Wp, h->agg, h->carry, h->sync_words, h->wait_limit,
                              h->test_unpublished, h->st, h->stream);
    else
      e = bsf_launch_vscan(h->precision, h->n, skews[i], false, h->S, h->pitch, Hb, h->Wp,
                           h->scan_chunk, h->agg, h->carry, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "vertical scan");
  }
  h->have_S = true;
  h->S_R = h->R;
  h->S_elem = h->elem;
  h->S_q = h->q;
  h->S_row0 = row0;
  h->S_rows = rows;
  h->S_dirset = h->dirset;
  return BSF_OK;
}

}  // namespace

extern "C" {

int bsf_create(bsf_t* out, int H, int W, int N, int n, int boundary, int max_reach) {
  if (!out) return BSF_EINVAL;
  *out = nullptr;
  if (H <= 0 || W <= 0 || N != 4 || n < 1 || n > 3 || boundary < BSF_ZERO ||
      boundary > BSF_SYMMETRIC || max_reach < -1)
    return BSF_EINVAL;
  if ((long long)H * W > (1LL << 31)) return BSF_EINVAL;
  bsf_t h = new (std::nothrow) bsf_ctx();
  if (!h) return BSF_ENOMEM;
  h->H = H; h->W = W; h->N = N; h->n = n; h->boundary = boundary;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return BSF_ECUDA; }
  if (max_reach >= 0) {
    h->R = max_reach > 3 * n ? max_reach : 3 * n;
    h->R_fixed = true;
  }
  cudaError_t e = cudaMalloc(&h->st, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMemset(h->st, 0, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMalloc(&h->Lf, (size_t)H * W * sizeof(ushort4));
  if (e == cudaSuccess && h->R_fixed && ensure_workspace(h) != BSF_OK) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    bsf_destroy(h);
    return e == cudaErrorMemoryAllocation ? BSF_ENOMEM : BSF_ECUDA;
  }
  *out = h;
  return BSF_OK;
}

void bsf_destroy(bsf_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_workspace(h);
  if (h->tp_fields) cudaFree(h->tp_fields);
  if (h->tp_g) cudaFree(h->tp_g);
  if (h->tp_min) cudaFree(h->tp_min);
  if (h->hs_img) cudaFree(h->hs_img);
  if (h->hs_cov) cudaFree(h->hs_cov);
  if (h->hs_out) cudaFree(h->hs_out);
  if (h->hev_ready)
    for (auto& e : h->hev) cudaEventDestroy(e);
  if (h->hgraph) cudaGraphExecDestroy(h->hgraph);
  if (h->s_cap) cudaStreamDestroy(h->s_cap);
  if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
  if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
  if (h->ev) {
    for (int i = 0; i < 2 * bsf_ctx::kMaxRec; ++i) cudaEventDestroy(h->ev[i]);
    delete[] h->ev;
  }
  if (h->Lf) cudaFree(h->Lf);
  if (h->st) cudaFree(h->st);
  delete h;
}

int bsf_set_stream(bsf_t h, void* stream) {
  if (!h) return BSF_EINVAL;
  h->stream = (cudaStream_t)stream;
  return BSF_OK;
}

int bsf_set_precision(bsf_t h, int mode, int frac_bits) {
  if (!h) return BSF_EINVAL;
  if (mode != BSF_FIX && mode != BSF_FIX32 && mode != BSF_FIX64 && mode != BSF_FIX128 &&
      mode != BSF_F64ACC && mode != BSF_F32KAHAN)
    return fail(h, BSF_EINVAL, "bad precision mode %d", mode);
  const int qmax = mode == BSF_FIX32 ? 30 : (mode == BSF_FIX64 || mode == BSF_FIX ? 62 : 100);
  if (frac_bits < -1 || frac_bits > qmax)
    return fail(h, BSF_EINVAL, "frac_bits %d outside [-1, %d]", frac_bits, qmax);
  const int eff = mode == BSF_FIX ? (is_fixed(h->precision) ? h->precision : BSF_FIX64) : mode;
  if (eff != h->precision) h->have_S = false;
  h->precision = eff;
  h->prec_auto = mode == BSF_FIX;
  h->frac_req = frac_bits;
  return BSF_OK;
}

int bsf_set_value_bound(bsf_t h, double max_abs) {
  if (!h) return BSF_EINVAL;
  if (!(max_abs >= 0.0) || std::isinf(max_abs)) return fail(h, BSF_EINVAL, "bad value bound");
  h->has_bound = true;
  h->value_bound = max_abs;
  return BSF_OK;
}

int bsf_set_step_rule(bsf_t h, int rule) {
  if (!h) return BSF_EINVAL;
  if (rule != BSF_STEP_D1 && rule != BSF_STEP_D1_PAPER && rule != BSF_STEP_D2 && rule != BSF_STEP_SAMPLED)
    return fail(h, BSF_EINVAL, "bad step rule %d", rule);
  if (rule == BSF_STEP_SAMPLED && h->n != 1) return fail(h, BSF_EINVAL, "the sampled box spline is of order 1");
  if (rule == BSF_STEP_D2 && h->n > 2) return fail(h, BSF_EINVAL, "continuous steps need n <= 2");
  if (rule != h->step_rule) h->planned = false;  // the mass bound differs between rules
  h->step_rule = rule;
  return BSF_OK;
}

int bsf_set_option(bsf_t h, int option, long long value) {
  if (!h) return BSF_EINVAL;
  switch (option) {
    case BSF_OPT_SCAN_MODE:
      if (value != BSF_SCAN_LOOKBACK && value != BSF_SCAN_THREE_PHASE)
        return fail(h, BSF_EINVAL, "bad scan mode %lld", value);
      h->scan_mode = (int)value;
      return BSF_OK;
    case BSF_OPT_WAIT_LIMIT:
      if (value < 0 || value > (1LL << 30)) return fail(h, BSF_EINVAL, "bad wait limit %lld", value);
      h->wait_limit = (int)value;
      return BSF_OK;
    case BSF_OPT_SCAN_CHUNK:
      if (value < kScanChunkMin || value > 4096) return fail(h, BSF_EINVAL, "bad scan chunk %lld", value);
      h->scan_chunk = (int)value;
      return BSF_OK;
    case BSF_OPT_SCAN_SHORT_TILES:
      h->short_tiles = value != 0;
      return BSF_OK;
    case BSF_OPT_TEST_UNPUBLISHED:
      h->test_unpublished = value != 0;
      return BSF_OK;
    case BSF_OPT_PLAN_UNION:
      h->plan_union = value != 0;
      return BSF_OK;
    case BSF_OPT_DIRECTIONS:
      if (value < BSF_DIRS_CARTESIAN || value > BSF_DIRS_PAIR)
        return fail(h, BSF_EINVAL, "bad direction set %lld", value);
      if (value != h->dirset) {
        h->dirset = (int)value;
        h->planned = false;  // reach and mass differ between the sets
        h->have_S = false;
        h->steps_current = false;
      }
      return BSF_OK;
    case BSF_OPT_TILES:
      if (value != 0 && value != 1) return fail(h, BSF_EINVAL, "bad tiles option %lld", value);
      h->tiles = (int)value;
      return BSF_OK;
    case BSF_OPT_HOST_BANDS:
      if (value < 1 || value > bsf_ctx::kHostBands) return fail(h, BSF_EINVAL, "bad band count %lld", value);
      h->host_bands = (int)value;
      return BSF_OK;
    default:
      return fail(h, BSF_EINVAL, "unknown option %d", option);
  }
}

int bsf_plan(bsf_t h, const float* cov, int cov_kind) {
  if (!h) return BSF_EINVAL;
  return run_steps(h, cov, cov_kind, true);
}

int bsf_preintegrate(bsf_t h, const void* img, int dtype, long long ld) {
  if (!h) return BSF_EINVAL;
  return preintegrate_impl(h, img, dtype, ld, 0, h->H);
}

static int filter_impl(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                       int cov_kind, void* out, int out_dtype, long long ldo, int row0, int rows,
                       float* jac = nullptr, long long ldj = 0) {
  if (!h) return BSF_EINVAL;
  if (!out) return fail(h, BSF_EINVAL, "out is NULL");
  if (h->step_rule == BSF_STEP_D2) {
    const int rc = check_d2(h);
    if (rc) return rc;
  }
  if (h->step_rule == BSF_STEP_SAMPLED) {
    if (h->precision != BSF_FIX64 && h->precision != BSF_FIX128) {
      if (!(h->prec_auto && h->precision == BSF_FIX32))
        return fail(h, BSF_EINVAL, "the sampled box spline needs BSF_FIX64 or BSF_FIX128");
      h->precision = BSF_FIX64;  // BSF_FIX: chosen again at the pre-integration, 64 bits at least
      h->have_S = false;
    }
    if (jac) return fail(h, BSF_EINVAL, "the sampled box spline has no Jacobian");
    const int minpad = h->dirset == BSF_DIRS_CARTESIAN ? kSampledMinPad : kSampledMinPadSecond;
    if (h->R >= 0 && h->R < minpad)
      return fail(h, BSF_EINVAL, "padding R = %d below %d, the reach of the sampled taps", h->R, minpad);
  }
  if (h->dirset != BSF_DIRS_CARTESIAN) {
    if (h->step_rule == BSF_STEP_D2)
      return fail(h, BSF_EINVAL, "the second direction set: integer or sampled steps only");
    if (!is_fixed(h->precision)) return fail(h, BSF_EINVAL, "the second direction set needs fixed point");
  }
  if (out_dtype != BSF_F32 && out_dtype != BSF_F64) return fail(h, BSF_EINVAL, "bad out dtype %d", out_dtype);
  if (ldo < h->W) return fail(h, BSF_EINVAL, "ldo %lld < W %d", ldo, h->W);
  if (row0 < 0 || rows <= 0 || row0 + rows > h->H) return fail(h, BSF_EINVAL, "bad row band");
  int rc = check_cov_kind(h, cov_kind);
  if (rc) return rc;
  if (!cov) return fail(h, BSF_EINVAL, "cov is NULL");
  // the step field itself is solved inside the stencil; a separate solve
  // runs only to plan R and the mass bound
  const bool need_plan = h->R < 0 || (img && h->frac_req < 0 && !h->planned);
  if (need_plan) {
    if ((rc = run_steps(h, cov, cov_kind, true))) return rc;
  }
  if ((rc = reset_counters(h, true, false))) return rc;
  // one fused kernel of restarted tiles, when a tile fits in shared memory
  if (img && h->tiles && !jac && (h->step_rule == BSF_STEP_D1 || h->step_rule == BSF_STEP_D1_PAPER) &&
      h->R >= 0 && (h->dirset == BSF_DIRS_CARTESIAN || is_fixed(h->precision))) {
    if (dtype != BSF_U8 && dtype != BSF_F32 && dtype != BSF_F64)
      return fail(h, BSF_EINVAL, "bad image dtype %d", dtype);
    if (ld < h->W) return fail(h, BSF_EINVAL, "ld %lld < W %d", ld, h->W);
    if ((rc = resolve_q(h, img, dtype, ld))) return rc;  // may choose the element (BSF_FIX)
    if (!h->max_smem) {
      int v = 0;
      BSF_CUDA(h, cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
      h->max_smem = v;
    }
    const int TT = bsf_tile_size(h->precision, h->R, h->max_smem, h->dirset == BSF_DIRS_PAIR ? 2 : 1);
    if (TT > 0) {
      if ((rc = reset_counters(h, false, true))) return rc;
      cudaError_t e;
      {
        PhaseTimer t(h, BSF_PHASE_TILES);
        e = bsf_launch_tiles(h->precision, h->n, h->dirset, img, dtype, ld, h->H, h->W, h->R, h->boundary, row0, rows,
                             TT, h->q, cov, cov_kind, h->step_rule, out, out_dtype, ldo, h->st, h->stream);
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "tile filter");
      h->have_S = false;  // no running sums are kept
      h->last_cov = cov;
      h->last_kind = cov_kind;
      h->steps_current = false;
      return BSF_OK;
    }
  }
  if (img) {
    if ((rc = preintegrate_impl(h, img, dtype, ld, row0, rows))) return rc;
  } else if (!h->have_S || h->S_R != h->R || h->S_elem != h->elem || h->S_row0 != row0 ||
             h->S_rows != rows || h->S_dirset != h->dirset) {
    return fail(h, BSF_ESTATE, "img is NULL and no matching pre-integration is held");
  }
  cudaError_t e;
  {
    PhaseTimer t(h, BSF_PHASE_STENCIL);
    if (h->step_rule == BSF_STEP_D2)
      e = bsf_launch_stencil_d2(h->precision, h->n, jac ? 1 : 0, h->S, h->pitch, h->R, cov, cov_kind,
                                h->H, h->W, row0, rows, h->S_q, out, out_dtype, ldo, jac, ldj,
                                (long long)rows * ldj, nullptr, 0, h->st, h->stream);
    else if (h->step_rule == BSF_STEP_SAMPLED)
      e = bsf_launch_stencil_sampled(h->precision, h->dirset, h->S, h->S2, h->pitch, h->R, cov, cov_kind, h->H,
                                     h->W, row0, rows, h->S_q, out, out_dtype, ldo, h->st, h->stream);
    else if (h->dirset == BSF_DIRS_CARTESIAN)
      e = bsf_launch_stencil_d1_ex(h->precision, h->n, h->S, h->pitch, h->R, cov, cov_kind,
                                   h->step_rule, h->H, h->W, row0, rows, h->S_q, out, out_dtype, ldo,
                                   h->st, h->stream, img != nullptr && !h->profiling);
    else
      e = bsf_launch_stencil_sets(h->precision, h->n, h->dirset, h->S, h->S2, h->pitch, h->R, cov,
                                  cov_kind, h->step_rule, h->H, h->W, row0, rows, h->S_q, out,
                                  out_dtype, ldo, h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "stencil");
  if (h->last_cov != cov || h->last_kind != cov_kind) h->steps_current = false;
  h->last_cov = cov;
  h->last_kind = cov_kind;
  return BSF_OK;
}

int bsf_filter(bsf_t h, const void* img, int dtype, long long ld, const float* cov, int cov_kind,
               void* out, int out_dtype, long long ldo) {
  if (!h) return BSF_EINVAL;
  return filter_impl(h, img, dtype, ld, cov, cov_kind, out, out_dtype, ldo, 0, h->H);
}

// (Re)allocate a device staging buffer of at least `bytes`.
static int ensure_staging(bsf_t h, void*& buf, size_t& have, size_t bytes) {
  if (have >= bytes) return BSF_OK;
  BSF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (buf) cudaFree(buf);
  buf = nullptr;
  have = 0;
  BSF_CUDA(h, cudaMalloc(&buf, bytes));
  have = bytes;
  return BSF_OK;
}

// Output rows [y0, y0 + rows) from the whole image's running sums (the
// stencil reads S from row y0 of the padded domain on).
static cudaError_t stencil_band(bsf_t h, const float* cov, int cov_kind, int y0, int rows, void* out,
                                int out_dtype, long long ldo) {
  const void* S = static_cast<const char*>(h->S) + (size_t)y0 * h->pitch * h->elem;
  if (h->dirset != BSF_DIRS_CARTESIAN) {
    const void* S2 = h->S2 ? static_cast<const char*>(h->S2) + (size_t)y0 * h->pitch * h->elem : nullptr;
    return bsf_launch_stencil_sets(h->precision, h->n, h->dirset, S, S2, h->pitch, h->R, cov, cov_kind,
                                   h->step_rule, h->H, h->W, y0, rows, h->S_q, out, out_dtype, ldo,
                                   h->st, h->stream);
  }
  if (h->step_rule == BSF_STEP_D2)
    return bsf_launch_stencil_d2(h->precision, h->n, 0, S, h->pitch, h->R, cov, cov_kind, h->H, h->W,
                                 y0, rows, h->S_q, out, out_dtype, ldo, nullptr, 0, 0, nullptr, 0,
                                 h->st, h->stream);
  if (h->step_rule == BSF_STEP_SAMPLED) {
    const void* S2 = h->S2 ? static_cast<const char*>(h->S2) + (size_t)y0 * h->pitch * h->elem : nullptr;
    return bsf_launch_stencil_sampled(h->precision, h->dirset, S, S2, h->pitch, h->R, cov, cov_kind, h->H, h->W,
                                      y0, rows, h->S_q, out, out_dtype, ldo, h->st, h->stream);
  }
  return bsf_launch_stencil_d1(h->precision, h->n, S, h->pitch, h->R, cov, cov_kind, h->step_rule,
                               h->H, h->W, y0, rows, h->S_q, out, out_dtype, ldo, h->st, h->stream);
}

// The work of bsf_filter_host after the staging buffers exist: uploads on
// s_h2d, pre-integration and band stencils on h->stream, downloads on s_d2h.
static int enqueue_host_filter(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                               int cov_kind, void* out, int out_dtype, long long ldo, bool plan) {
  const int H = h->H, W = h->W;
  const size_t HW = (size_t)H * W;
  const size_t es = dtype == BSF_U8 ? 1 : (dtype == BSF_F32 ? 4 : 8), eo = out_dtype == BSF_F32 ? 4 : 8;
  const int K = H < h->host_bands ? H : h->host_bands;
  cudaEvent_t ev_img = h->hev[0];
  cudaEvent_t* ev_cov = h->hev + 1;
  cudaEvent_t* ev_out = h->hev + 1 + bsf_ctx::kHostBands;
  // the last band is a quarter of the others' height: only its stencil and
  // its download remain after the last upload
  const long long den = 4LL * (K - 1) + 1;
  auto band = [&](int k, int& y0, int& rows) {
    y0 = (int)(H * 4LL * k / den);
    rows = (k == K - 1 ? H : (int)(H * 4LL * (k + 1) / den)) - y0;
  };
  float* dcov = static_cast<float*>(h->hs_cov);
  int rc;
  // the image on the upload stream, and its pre-integration queued right
  // behind it; then the field band by band (the three planes of a band in one
  // two-dimensional copy)
  BSF_CUDA(h, cudaMemcpy2DAsync(h->hs_img, W * es, img, ld * es, W * es, H, cudaMemcpyHostToDevice,
                                h->s_h2d));
  BSF_CUDA(h, cudaEventRecord(ev_img, h->s_h2d));
  auto upload_field = [&]() -> int {
    for (int k = 0; k < K; ++k) {
      int y0, rows;
      band(k, y0, rows);
      BSF_CUDA(h, cudaMemcpy2DAsync(dcov + (size_t)y0 * W, HW * sizeof(float), cov + (size_t)y0 * W,
                                    HW * sizeof(float), (size_t)rows * W * sizeof(float), 3,
                                    cudaMemcpyHostToDevice, h->s_h2d));
      BSF_CUDA(h, cudaEventRecord(ev_cov[k], h->s_h2d));
    }
    return BSF_OK;
  };
  if (plan) {
    // a plan (first call) needs the whole field first
    if ((rc = upload_field())) return rc;
    BSF_CUDA(h, cudaStreamWaitEvent(h->stream, ev_cov[K - 1], 0));
    if ((rc = run_steps(h, dcov, cov_kind, true))) return rc;
    if ((rc = reset_counters(h, true, false))) return rc;
    BSF_CUDA(h, cudaStreamWaitEvent(h->stream, ev_img, 0));
    if ((rc = preintegrate_impl(h, h->hs_img, dtype, W, 0, H))) return rc;
  } else {
    if ((rc = reset_counters(h, true, false))) return rc;
    BSF_CUDA(h, cudaStreamWaitEvent(h->stream, ev_img, 0));
    if ((rc = preintegrate_impl(h, h->hs_img, dtype, W, 0, H))) return rc;
    if ((rc = upload_field())) return rc;
  }
  for (int k = 0; k < K; ++k) {
    int y0, rows;
    band(k, y0, rows);
    BSF_CUDA(h, cudaStreamWaitEvent(h->stream, ev_cov[k], 0));
    cudaError_t e;
    {
      PhaseTimer t(h, BSF_PHASE_STENCIL);
      e = stencil_band(h, dcov, cov_kind, y0, rows, static_cast<char*>(h->hs_out) + (size_t)y0 * W * eo,
                       out_dtype, W);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "stencil");
    BSF_CUDA(h, cudaEventRecord(ev_out[k], h->stream));
    // each finished band goes back while the next one is computed
    BSF_CUDA(h, cudaStreamWaitEvent(h->s_d2h, ev_out[k], 0));
    BSF_CUDA(h, cudaMemcpy2DAsync(static_cast<char*>(out) + (size_t)y0 * ldo * eo, ldo * eo,
                                  static_cast<const char*>(h->hs_out) + (size_t)y0 * W * eo, W * eo,
                                  W * eo, rows, cudaMemcpyDeviceToHost, h->s_d2h));
  }
  return BSF_OK;
}

int bsf_filter_host(bsf_t h, const void* img, int dtype, long long ld, const float* cov, int cov_kind,
                    void* out, int out_dtype, long long ldo) {
  if (!h) return BSF_EINVAL;
  if (!img || !cov || !out) return fail(h, BSF_EINVAL, "NULL img, cov or out");
  if (dtype != BSF_U8 && dtype != BSF_F32 && dtype != BSF_F64)
    return fail(h, BSF_EINVAL, "bad image dtype %d", dtype);
  if (out_dtype != BSF_F32 && out_dtype != BSF_F64) return fail(h, BSF_EINVAL, "bad out dtype %d", out_dtype);
  if (ld < h->W || ldo < h->W) return fail(h, BSF_EINVAL, "leading dimension < W");
  int rc = check_cov_kind(h, cov_kind);
  if (rc) return rc;
  if (h->step_rule == BSF_STEP_D2 && (rc = check_d2(h))) return rc;
  const size_t HW = (size_t)h->H * h->W;
  const size_t es = dtype == BSF_U8 ? 1 : (dtype == BSF_F32 ? 4 : 8), eo = out_dtype == BSF_F32 ? 4 : 8;
  if ((rc = ensure_staging(h, h->hs_img, h->hs_img_bytes, HW * es))) return rc;
  if ((rc = ensure_staging(h, h->hs_cov, h->hs_cov_bytes, 3 * HW * sizeof(float)))) return rc;
  if ((rc = ensure_staging(h, h->hs_out, h->hs_out_bytes, HW * eo))) return rc;
  if (!h->s_h2d) BSF_CUDA(h, cudaStreamCreateWithFlags(&h->s_h2d, cudaStreamNonBlocking));
  if (!h->s_d2h) BSF_CUDA(h, cudaStreamCreateWithFlags(&h->s_d2h, cudaStreamNonBlocking));
  if (!h->s_cap) BSF_CUDA(h, cudaStreamCreateWithFlags(&h->s_cap, cudaStreamNonBlocking));
  if (!h->hev_ready) {
    for (auto& e : h->hev) BSF_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->hev_ready = true;
  }
  // the previous call's output copies must be done before the staging buffers are reused
  BSF_CUDA(h, cudaStreamSynchronize(h->s_d2h));
  const bool plan = h->R < 0 || (h->frac_req < 0 && !h->planned);
  // q known without a device reduction (which synchronises)?
  const bool q_known = !is_fixed(h->precision) || h->frac_req >= 0 || dtype == BSF_U8 || h->has_bound;
  if (plan || !q_known || h->profiling) {
    if ((rc = enqueue_host_filter(h, img, dtype, ld, cov, cov_kind, out, out_dtype, ldo, plan))) return rc;
  } else {
    if ((rc = resolve_q(h, nullptr, dtype, ld))) return rc;  // host arithmetic only here
    if ((rc = ensure_workspace(h))) return rc;
    const long long key[18] = {(long long)img, (long long)cov, (long long)out, dtype, ld, ldo, out_dtype,
                               cov_kind, h->host_bands, h->step_rule, h->precision, h->q, h->R,
                               (long long)h->S, h->pitch, h->scan_chunk, h->dirset, (long long)h->S2};
    if (!h->hgraph || std::memcmp(key, h->hkey, sizeof key) != 0) {
      if (h->hgraph) {
        cudaGraphExecDestroy(h->hgraph);
        h->hgraph = nullptr;
      }
      // capture on a private stream (the legacy default stream cannot be
      // captured); the copy streams join through events
      cudaStream_t user = h->stream;
      h->stream = h->s_cap;
      cudaEvent_t fork = h->hev[2 * bsf_ctx::kHostBands + 1];
      cudaEvent_t j1 = h->hev[2 * bsf_ctx::kHostBands + 2], j2 = h->hev[2 * bsf_ctx::kHostBands + 3];
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(h->s_cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) e = cudaEventRecord(fork, h->s_cap);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_h2d, fork, 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_d2h, fork, 0);
      int rc2 = e == cudaSuccess ? enqueue_host_filter(h, img, dtype, ld, cov, cov_kind, out, out_dtype,
                                                       ldo, false)
                                 : BSF_OK;
      if (e == cudaSuccess) e = cudaEventRecord(j1, h->s_h2d);
      if (e == cudaSuccess) e = cudaEventRecord(j2, h->s_d2h);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_cap, j1, 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_cap, j2, 0);
      const cudaError_t ec = cudaStreamEndCapture(h->s_cap, &graph);
      h->stream = user;
      if (e == cudaSuccess) e = ec;
      if (rc2) {
        if (graph) cudaGraphDestroy(graph);
        return rc2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->hgraph, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(h, e, "host-buffer graph");
      std::memcpy(h->hkey, key, sizeof key);
    }
    BSF_CUDA(h, cudaGraphLaunch(h->hgraph, h->stream));
  }
  h->last_cov = nullptr;  // the staged field is overwritten by the next call
  h->steps_current = false;
  BSF_CUDA(h, cudaStreamSynchronize(h->s_d2h));
  BSF_CUDA(h, cudaStreamSynchronize(h->stream));
  return BSF_OK;
}

int bsf_filter_two_pass(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                        int cov_kind, double frac, void* out, int out_dtype, long long ldo,
                        float* sigma2) {
  if (!h) return BSF_EINVAL;
  if (!img || !cov || !out) return fail(h, BSF_EINVAL, "NULL img, cov or out");
  if (!(frac > 0.0 && frac < 1.0)) return fail(h, BSF_EINVAL, "frac must lie in (0, 1)");
  if (h->step_rule == BSF_STEP_D2 || h->step_rule == BSF_STEP_SAMPLED)
    return fail(h, BSF_EINVAL, "two passes: integer steps only");
  int rc = check_cov_kind(h, cov_kind);
  if (rc) return rc;
  const size_t HW = (size_t)h->H * h->W;
  if (!h->tp_fields) {
    BSF_CUDA(h, cudaStreamSynchronize(h->stream));
    BSF_CUDA(h, cudaMalloc(&h->tp_fields, 6 * HW * sizeof(float)));
    BSF_CUDA(h, cudaMalloc(&h->tp_g, HW * sizeof(float)));
    BSF_CUDA(h, cudaMalloc(&h->tp_min, 2 * sizeof(unsigned long long)));
  }
  float* iso = h->tp_fields;
  float* res = h->tp_fields + 3 * HW;
  cudaError_t e;
  {
    PhaseTimer t(h, BSF_PHASE_STEPS);
    e = bsf_launch_cov_split(cov, cov_kind, h->H, h->W, frac, h->tp_min, iso, res, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "field split");
  if (h->R < 0 || (h->frac_req < 0 && !h->planned)) {
    // the padding and the mass bound must cover both fields
    const bool was_union = h->plan_union;
    h->plan_union = true;
    h->planned = false;
    rc = run_steps(h, iso, BSF_COV_C, true);
    if (!rc) rc = run_steps(h, res, BSF_COV_C, true);
    h->plan_union = was_union;
    if (rc) return rc;
  }
  if ((rc = filter_impl(h, img, dtype, ld, iso, BSF_COV_C, h->tp_g, BSF_F32, h->W, 0, h->H))) return rc;
  if ((rc = filter_impl(h, h->tp_g, BSF_F32, h->W, res, BSF_COV_C, out, out_dtype, ldo, 0, h->H)))
    return rc;
  if (sigma2) {
    unsigned long long b = 0;
    BSF_CUDA(h, cudaMemcpyAsync(&b, h->tp_min, sizeof b, cudaMemcpyDeviceToHost, h->stream));
    BSF_CUDA(h, cudaStreamSynchronize(h->stream));
    double m;
    std::memcpy(&m, &b, sizeof m);
    *sigma2 = (float)(frac * m);
  }
  return BSF_OK;
}

int bsf_filter_rows(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                    int cov_kind, void* out, int out_dtype, long long ldo, int y0, int y1) {
  if (!h) return BSF_EINVAL;
  if (!img) return fail(h, BSF_EINVAL, "img is NULL");
  return filter_impl(h, img, dtype, ld, cov, cov_kind, out, out_dtype, ldo, y0, y1 - y0);
}

int bsf_filter_jacobian(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                        int cov_kind, void* out, int out_dtype, long long ldo, float* jac,
                        long long ldj) {
  if (!h) return BSF_EINVAL;
  if (h->step_rule != BSF_STEP_D2) return fail(h, BSF_EINVAL, "the Jacobian needs BSF_STEP_D2");
  if (!jac) return fail(h, BSF_EINVAL, "jac is NULL");
  if (ldj < h->W) return fail(h, BSF_EINVAL, "ldj %lld < W %d", ldj, h->W);
  if (out_dtype != BSF_F32) return fail(h, BSF_EINVAL, "the Jacobian comes with float32 output");
  return filter_impl(h, img, dtype, ld, cov, cov_kind, out, out_dtype, ldo, 0, h->H, jac, ldj);
}

int bsf_jacobian_vjp(bsf_t h, const float* gout, long long ldg, const float* jac, long long ldj,
                     float* gcov) {
  if (!h) return BSF_EINVAL;
  if (!gout || !jac || !gcov) return fail(h, BSF_EINVAL, "NULL gout, jac or gcov");
  if (ldg < h->W || ldj < h->W) return fail(h, BSF_EINVAL, "leading dimension < W");
  PhaseTimer t(h, BSF_PHASE_VJP);
  cudaError_t e = bsf_launch_jacobian_vjp(gout, ldg, jac, ldj, gcov, h->H, h->W, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "jacobian vjp");
  return BSF_OK;
}

// Width of the backward's adjoint sums: 128 bits for the continuous steps and
// for contexts whose running sums are 128 bits (kernel masses beyond the reach
// of 64-bit weights), 64 bits otherwise.  The forward's element type plays no
// other part in the backward (it reads no running sums).
static int grad_elem(bsf_t h) {
  return h->step_rule == BSF_STEP_D2 || h->precision == BSF_FIX128 ? 16 : 8;
}
static int grad_prec(int be) { return be == 16 ? BSF_FIX128 : BSF_FIX64; }
static int grad_q_max(int be) { return be == 16 ? 126 : 100; }

// G (adjoint running sums), Gx (row-folded) and the chunk states of the
// reversed vertical sums, for the whole padded domain, in elements of be bytes.
static int ensure_backward_workspace(bsf_t h, int be) {
  if (h->R < 0) return fail(h, BSF_ESTATE, "padding unknown: plan or filter first");
  int rc;
  if ((rc = ensure_workspace(h))) return rc;
  const size_t G_bytes = (size_t)h->pitch * h->Hp * be, Gx_bytes = (size_t)h->Hp * h->W * be;
  const int nchunks = (h->Hp + kScanChunkMin - 1) / kScanChunkMin;
  const size_t bagg_bytes = (size_t)nchunks * h->n * (size_t)(h->Wp + h->Hp - 1) * be;
  if (h->G_bytes != G_bytes || h->Gx_bytes != Gx_bytes || h->bagg_bytes != bagg_bytes) {
    BSF_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->G) cudaFree(h->G);
    if (h->Gx) cudaFree(h->Gx);
    if (h->bagg) cudaFree(h->bagg);
    h->G = h->Gx = h->bagg = nullptr;
    h->G_bytes = h->Gx_bytes = h->bagg_bytes = 0;
    BSF_CUDA(h, cudaMalloc(&h->G, G_bytes));
    BSF_CUDA(h, cudaMalloc(&h->Gx, Gx_bytes));
    BSF_CUDA(h, cudaMalloc(&h->bagg, bagg_bytes));
    h->G_bytes = G_bytes;
    h->Gx_bytes = Gx_bytes;
    h->bagg_bytes = bagg_bytes;
  }
  return BSF_OK;
}

// Reversed n-fold sums of G over Hb padded rows: d4, d2, d3 (three-phase, or
// the look-back scan for 64-bit sums of a 64-bit context), then the rows.
static int backward_sums(bsf_t h, int be, int Hb) {
  cudaError_t e = cudaSuccess;
  const int skews[3] = {-1, 1, 0};  // transposes in reverse order: d4, d2, d3
  const bool lb = h->scan_mode == BSF_SCAN_LOOKBACK && be == 8 && h->elem == 8 && Hb == h->Hp;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    if (lb)
      e = bsf_launch_vscan_lb(BSF_FIX64, h->n, skews[i], true, h->short_tiles != 0, h->G, h->pitch, h->Hp,
                              h->Wp, h->agg, h->carry, h->sync_words, h->wait_limit, 0, h->st, h->stream);
    else
      e = bsf_launch_vscan(grad_prec(be), h->n, skews[i], true, h->G, h->pitch, Hb, h->Wp, h->scan_chunk,
                           h->bagg, nullptr, h->stream);
  }
  if (e == cudaSuccess) e = bsf_launch_suffix_rows(be, h->n, h->G, h->pitch, Hb, h->Wp, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "backward running sums");
  return BSF_OK;
}

int bsf_grad_frac_bits(double max_abs_gout) { return bsf_grad_q_host(max_abs_gout); }

int bsf_grad_frac_bits_of(bsf_t h, double max_abs_gout) {
  if (!h) return BSF_EINVAL;
  return grad_elem(h) == 16 ? bsf_grad_q_host_wide(max_abs_gout) : bsf_grad_q_host(max_abs_gout);
}

int bsf_grad_absmax_rows(bsf_t h, const float* gout, long long ldg, int y0, int y1, float* result) {
  if (!h) return BSF_EINVAL;
  if (!gout || !result) return fail(h, BSF_EINVAL, "NULL gout or result");
  if (ldg < h->W || y0 < 0 || y1 <= y0 || y1 > h->H) return fail(h, BSF_EINVAL, "bad rows or ldg");
  BSF_CUDA(h, cudaMemsetAsync(&h->st->max_absg_bits, 0, sizeof(unsigned), h->stream));
  cudaError_t e = bsf_launch_gabsmax(gout + (long long)y0 * ldg, ldg, y1 - y0, h->W, h->st, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "gradient maximum");
  int rc = read_status(h);
  if (rc) return rc;
  const unsigned b = h->host_st.max_absg_bits;
  std::memcpy(result, &b, sizeof b);
  return BSF_OK;
}

int bsf_filter_backward_rows(bsf_t h, const float* gout, long long ldg, const float* cov,
                             int cov_kind, int y0, int y1, int grad_bits, long long* acc,
                             long long lda) {
  if (!h) return BSF_EINVAL;
  int rc = check_cov_kind(h, cov_kind);
  if (rc) return rc;
  if (h->step_rule == BSF_STEP_SAMPLED) return fail(h, BSF_EINVAL, "the sampled box spline: forward only");
  if (h->step_rule == BSF_STEP_D2 && (rc = check_d2(h))) return rc;
  if (h->dirset != BSF_DIRS_CARTESIAN) return fail(h, BSF_EINVAL, "backward: Cartesian direction set only");
  if (!gout || !cov || !acc) return fail(h, BSF_EINVAL, "NULL gout, cov or acc");
  if (ldg < h->W || lda < h->W) return fail(h, BSF_EINVAL, "leading dimension < W");
  if (y0 < 0 || y1 <= y0 || y1 > h->H) return fail(h, BSF_EINVAL, "bad row band");
  const int be = grad_elem(h);
  if (grad_bits < 0 || grad_bits > grad_q_max(be))
    return fail(h, BSF_EINVAL, "grad_bits outside [0, %d]", grad_q_max(be));
  if ((rc = ensure_backward_workspace(h, be))) return rc;
  if (h->R > h->H) return fail(h, BSF_EINVAL, "band backward needs R <= H");
  const int rows = y1 - y0, Hb = rows + 2 * h->R;
  const int a0 = y0 - h->R > 0 ? y0 - h->R : 0, a1 = y1 + h->R < h->H ? y1 + h->R : h->H;
  if ((rc = reset_counters(h, true, false))) return rc;
  cudaError_t e;
  {
    PhaseTimer t(h, BSF_PHASE_BWD_SCATTER);
    BSF_CUDA(h, cudaMemsetAsync(h->G, 0, (size_t)h->pitch * Hb * be, h->stream));
    if (h->step_rule == BSF_STEP_D2)
      e = bsf_launch_scatter_d2(h->n, h->G, h->pitch, h->R, cov, cov_kind, gout, ldg, h->H, h->W, y0, rows,
                                grad_bits, h->st, h->stream);
    else
      e = bsf_launch_scatter_d1(h->n, be, h->G, h->pitch, h->R, cov, cov_kind, h->step_rule, gout, ldg,
                                h->H, h->W, y0, rows, grad_bits, h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "band scatter");
  {
    PhaseTimer t(h, BSF_PHASE_BWD_SCANS);
    if ((rc = backward_sums(h, be, Hb))) return rc;
  }
  {
    PhaseTimer t(h, BSF_PHASE_BWD_FOLD);
    e = bsf_launch_fold_band(be, h->G, h->pitch, Hb, h->H, h->W, h->R, y0, h->boundary, h->Gx, a0, a1,
                             acc, lda, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "band fold");
  return BSF_OK;
}

int bsf_grad_finalize(bsf_t h, const long long* acc, long long lda, int rows, int grad_bits,
                      float* gimg, long long ldgi) {
  if (!h) return BSF_EINVAL;
  if (!acc || !gimg) return fail(h, BSF_EINVAL, "NULL acc or gimg");
  if (lda < h->W || ldgi < h->W || rows <= 0 || rows > h->H)
    return fail(h, BSF_EINVAL, "bad rows or leading dimension");
  const int be = grad_elem(h);
  if (grad_bits < 0 || grad_bits > grad_q_max(be))
    return fail(h, BSF_EINVAL, "grad_bits outside [0, %d]", grad_q_max(be));
  cudaError_t e = bsf_launch_grad_finalize(be, acc, lda, rows, h->W, grad_bits, gimg, ldgi, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "gradient finalize");
  return BSF_OK;
}

int bsf_grad_halo_add(bsf_t h, long long* acc, long long lda, const long long* halo, long long ldh,
                      int rows) {
  if (!h) return BSF_EINVAL;
  if (!acc || !halo) return fail(h, BSF_EINVAL, "NULL acc or halo");
  if (lda < h->W || ldh < h->W || rows <= 0 || rows > h->H)
    return fail(h, BSF_EINVAL, "bad rows or leading dimension");
  cudaError_t e = bsf_launch_add_rows(grad_elem(h), acc, lda, halo, ldh, rows, h->W, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "halo add");
  return BSF_OK;
}

// Continuous steps: gcov = gout * d out / d plane (from the held running sums),
// and/or the image gradient through uint128 adjoint sums.
static int backward_d2(bsf_t h, const float* gout, long long ldg, const float* cov, int cov_kind,
                       float* gimg, long long ldgi, float* gcov) {
  int rc = check_d2(h);
  if (rc) return rc;
  if (!gcov && !gimg) return fail(h, BSF_EINVAL, "continuous steps: gimg and gcov are NULL");
  if (h->R < 0) return fail(h, BSF_ESTATE, "padding unknown: plan or filter first");
  if ((rc = reset_counters(h, true, false))) return rc;
  cudaError_t e = cudaSuccess;
  if (gcov) {
    if (!h->have_S || h->S_R != h->R || h->S_elem != h->elem || h->S_row0 != 0 || h->S_rows != h->H)
      return fail(h, BSF_ESTATE, "no whole-image pre-integration is held");
    PhaseTimer t(h, BSF_PHASE_VJP);
    e = bsf_launch_stencil_d2(h->precision, h->n, 2, h->S, h->pitch, h->R, cov, cov_kind, h->H, h->W,
                              0, h->H, h->S_q, nullptr, BSF_F32, h->W, gcov, h->W,
                              (long long)h->H * h->W, gout, ldg, h->st, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "continuous-step vjp");
  }
  if (!gimg) return BSF_OK;
  // the image gradient reads no running sums: 128-bit adjoint sums whatever
  // the forward's element type
  if ((rc = ensure_backward_workspace(h, 16))) return rc;
  {
    PhaseTimer t(h, BSF_PHASE_BWD_SCATTER);
    BSF_CUDA(h, cudaMemsetAsync(&h->st->max_absg_bits, 0, sizeof(unsigned), h->stream));
    BSF_CUDA(h, cudaMemsetAsync(h->G, 0, h->G_bytes, h->stream));
    e = bsf_launch_gabsmax(gout, ldg, h->H, h->W, h->st, h->stream);
    if (e == cudaSuccess)
      e = bsf_launch_scatter_d2(h->n, h->G, h->pitch, h->R, cov, cov_kind, gout, ldg, h->H, h->W, 0, h->H, -1,
                                h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "continuous-step scatter");
  {
    PhaseTimer t(h, BSF_PHASE_BWD_SCANS);
    if ((rc = backward_sums(h, 16, h->Hp))) return rc;
  }
  {
    PhaseTimer t(h, BSF_PHASE_BWD_FOLD);
    e = bsf_launch_fold128(h->G, h->pitch, h->Hp, h->H, h->W, h->R, h->boundary, h->Gx, gimg, ldgi,
                           h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "continuous-step fold");
  return BSF_OK;
}

int bsf_filter_backward(bsf_t h, const float* gout, long long ldg, const float* cov, int cov_kind,
                        float* gimg, long long ldgi, float* gcov) {
  if (!h) return BSF_EINVAL;
  int rc = check_cov_kind(h, cov_kind);
  if (rc) return rc;
  if (h->dirset != BSF_DIRS_CARTESIAN) return fail(h, BSF_EINVAL, "backward: Cartesian direction set only");
  if (h->step_rule == BSF_STEP_SAMPLED) return fail(h, BSF_EINVAL, "the sampled box spline: forward only");
  if (h->step_rule == BSF_STEP_D2) {
    if (!gout || !cov) return fail(h, BSF_EINVAL, "NULL gout or cov");
    if (ldg < h->W || (gimg && ldgi < h->W)) return fail(h, BSF_EINVAL, "leading dimension < W");
    return backward_d2(h, gout, ldg, cov, cov_kind, gimg, ldgi, gcov);
  }
  if (!gout || !cov || !gimg) return fail(h, BSF_EINVAL, "NULL gout, cov or gimg");
  if (ldg < h->W || ldgi < h->W) return fail(h, BSF_EINVAL, "leading dimension < W");
  const int be = grad_elem(h);
  if ((rc = ensure_backward_workspace(h, be))) return rc;
  if ((rc = reset_counters(h, true, false))) return rc;
  cudaError_t e;
  {
    PhaseTimer t(h, BSF_PHASE_BWD_SCATTER);
    BSF_CUDA(h, cudaMemsetAsync(&h->st->max_absg_bits, 0, sizeof(unsigned), h->stream));
    BSF_CUDA(h, cudaMemsetAsync(h->G, 0, h->G_bytes, h->stream));
    e = bsf_launch_gabsmax(gout, ldg, h->H, h->W, h->st, h->stream);
    if (e == cudaSuccess)
      e = bsf_launch_scatter_d1(h->n, be, h->G, h->pitch, h->R, cov, cov_kind, h->step_rule, gout, ldg, h->H,
                                h->W, 0, h->H, -1, h->st, h->stream, true);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "backward scatter");
  {
    PhaseTimer t(h, BSF_PHASE_BWD_SCANS);
    if ((rc = backward_sums(h, be, h->Hp))) return rc;
  }
  {
    PhaseTimer t(h, BSF_PHASE_BWD_FOLD);
    if (be == 16)
      e = bsf_launch_fold128(h->G, h->pitch, h->Hp, h->H, h->W, h->R, h->boundary, h->Gx, gimg, ldgi, h->st,
                             h->stream);
    else
      e = bsf_launch_fold(h->G, h->pitch, h->Hp, h->H, h->W, h->R, h->boundary, h->Gx, gimg, ldgi,
                          h->st, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "backward fold");
  if (gcov) BSF_CUDA(h, cudaMemsetAsync(gcov, 0, (size_t)3 * h->H * h->W * sizeof(float), h->stream));
  return BSF_OK;
}

int bsf_status(bsf_t h) {
  if (!h) return BSF_EINVAL;
  int rc = read_status(h);
  if (rc) return rc;
  const int err = h->host_st.err;
  BSF_CUDA(h, cudaMemsetAsync(&h->st->err, 0, sizeof(int), h->stream));
  BSF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (err) {
    fail(h, err, "device status %d (clamped %u, non-finite %u, out of reach %u, overflow %u)", err,
         h->host_st.clamp_count, h->host_st.bad_count, h->host_st.range_count,
         h->host_st.overflow_count);
  }
  return err;
}

const char* bsf_last_error(bsf_t h) { return h ? h->msg : "NULL context"; }

int bsf_get_info(bsf_t h, bsf_info_t* info) {
  if (!h || !info) return BSF_EINVAL;
  std::memset(info, 0, sizeof *info);
  info->H = h->H; info->W = h->W; info->N = h->N; info->n = h->n;
  info->boundary = h->boundary;
  info->R = h->R;
  info->Hp = h->R >= 0 ? h->H + 2 * h->R : 0;
  info->Wp = h->R >= 0 ? h->W + 2 * h->R : 0;
  info->pitch = h->pitch;
  info->elem_bytes = (int)elem_bytes_of(h->precision);
  info->precision = h->precision;
  info->frac_bits = h->q;
  info->step_rule = h->step_rule;
  info->max_reach = h->plan_reach;
  info->max_mass = h->plan_mass;
  info->clamp_count = h->host_st.clamp_count;
  info->flags = h->host_st.clamp_count ? BSF_FLAG_CLAMPED : 0u;
  info->workspace_bytes = (long long)(h->S_bytes + 2 * h->scan_bytes + h->sync_bytes + h->G_bytes + h->Gx_bytes +
                                      h->bagg_bytes) +
                          (long long)h->H * h->W * (long long)sizeof(ushort4) + (long long)sizeof(DevStatus);
  info->grad_elem_bytes = grad_elem(h);
  return BSF_OK;
}

int bsf_copy_steps(bsf_t h, uint16_t* dst) {
  if (!h || !dst) return BSF_EINVAL;
  if (!h->last_cov) return fail(h, BSF_ESTATE, "no covariance seen yet");
  if (!h->steps_current) {  // solve the last field again (it must still be valid)
    const bool planned = h->planned;
    h->planned = true;  // bounded by the current R, no plan
    int rc = run_steps(h, h->last_cov, h->last_kind, false);
    h->planned = planned;
    if (rc) return rc;
  }
  const size_t HW = (size_t)h->H * h->W;
  for (int k = 0; k < 4; ++k) {
    BSF_CUDA(h, cudaMemcpy2DAsync(dst + k * HW, sizeof(uint16_t),
                                  reinterpret_cast<const char*>(h->Lf) + k * sizeof(uint16_t),
                                  sizeof(ushort4), sizeof(uint16_t), HW, cudaMemcpyDeviceToDevice,
                                  h->stream));
  }
  return BSF_OK;
}

int bsf_copy_preintegrated(bsf_t h, void* dst) {
  if (!h || !dst) return BSF_EINVAL;
  if (!h->have_S) return fail(h, BSF_ESTATE, "no pre-integration held");
  const size_t rows = (size_t)h->S_rows + 2 * h->S_R;
  BSF_CUDA(h, cudaMemcpy2DAsync(dst, (size_t)h->Wp * h->elem, h->S, (size_t)h->pitch * h->elem,
                                (size_t)h->Wp * h->elem, rows, cudaMemcpyDeviceToDevice, h->stream));
  if (h->S_dirset == BSF_DIRS_PAIR)  // the second set's sums follow the first's
    BSF_CUDA(h, cudaMemcpy2DAsync(static_cast<char*>(dst) + rows * h->Wp * h->elem, (size_t)h->Wp * h->elem,
                                  h->S2, (size_t)h->pitch * h->elem, (size_t)h->Wp * h->elem, rows,
                                  cudaMemcpyDeviceToDevice, h->stream));
  return BSF_OK;
}

int bsf_set_profiling(bsf_t h, int on) {
  if (!h) return BSF_EINVAL;
  if (on && !h->ev) {
    h->ev = new (std::nothrow) cudaEvent_t[2 * bsf_ctx::kMaxRec];
    if (!h->ev) return fail(h, BSF_ENOMEM, "event table");
    for (int i = 0; i < 2 * bsf_ctx::kMaxRec; ++i) BSF_CUDA(h, cudaEventCreate(&h->ev[i]));
  }
  h->profiling = on != 0;
  return BSF_OK;
}

int bsf_read_profile(bsf_t h, double* ms, int* count) {
  if (!h) return BSF_EINVAL;
  double acc[BSF_NUM_PHASES] = {0};
  int cnt[BSF_NUM_PHASES] = {0};
  if (h->nrec) BSF_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->nrec; ++i) {
    float t = 0.f;
    BSF_CUDA(h, cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]));
    acc[h->rec_phase[i]] += t;
    cnt[h->rec_phase[i]] += 1;
  }
  for (int p = 0; p < BSF_NUM_PHASES; ++p) {
    if (ms) ms[p] = acc[p];
    if (count) count[p] = cnt[p];
  }
  const int dropped = h->dropped;
  h->nrec = 0;
  h->dropped = 0;
  return dropped;
}

}  // extern "C"
