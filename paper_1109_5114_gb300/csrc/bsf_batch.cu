// Batched filtering of many images of uneven sizes (the C ABI's bsf_batch_*
// and bsf_filter_batched).  Every image keeps its own covariance field, padding
// R and scan chunk height; all images share one device arena and one q.
//
// A batched call issues one launch per phase for the whole batch -- row
// running sums, the agg and rescan kernels of the three vertical directions,
// the finite differences -- whose blocks find their image through per-phase
// block offsets, and can record those launches once in a CUDA graph and
// replay it.  The per-image mode runs the same kernels image by image (the
// baseline the batched form is measured against).
//
// BSF_BATCH_PERSISTENT runs the whole batch as one persistent launch
// (bsf_persistent.cu): resident blocks take work items -- rows, chunks of the
// vertical directions, tiles of the finite differences -- from one ticket
// counter, each item waiting (bounded) on a per-image counter of the phase
// before it; with BSF_BATCH_GRAPH that launch is recorded in a CUDA graph.
//
// The autotuner picks the scan chunk height per size class of the padded
// image (height classes up to 384, 768, 1536 rows and above), and the work
// item shapes of the persistent launch (padded rows per row item, rows of a
// finite-difference tile) and its blocks per SM, by timing the batch itself
// (coordinate descent over the candidates, the whole persistent launch as
// the objective); the choices can be kept in a text cache file between runs.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bsf_internal.h"

struct bsf_batch {
  int n = 2, boundary = BSF_SYMMETRIC, step_rule = BSF_STEP_D1;
  int frac_req = -1;
  bool has_bound = false;
  double value_bound = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;

  int B = 0;
  int dtype = BSF_F32, out_dtype = BSF_F32;
  int q = 0;
  std::vector<bsf_image_desc> descs;
  std::vector<BatchImage> imgs;
  std::vector<int> starts;        // kBatchPhases * (B + 1)
  int totals[kBatchPhases] = {0};
  BatchImage* d_imgs = nullptr;
  int* d_starts = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  DevStatus* st = nullptr;
  DevStatus host_st{};

  bool planned = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  int tune_chunk[4] = {0, 0, 0, 0};  // per height class; 0 = default
  std::string tune_cache;
  char msg[512] = "ok";

  // the persistent launch
  PersistentShape pshape{4, 1};
  int ctas_per_sm = 0;               // 0 = as many as fit
  int group_mb = 48;                 // running-sum bytes of one image group (0 = one group)
  int tuned_persist = 0;             // the shape and blocks came from the tuner or its cache
  int wait_limit = 1 << 22;          // polls of one wait before BSF_ETIMEOUT
  int test_withhold = 0;
  std::vector<PersistSegment> psegs;  // kPersistPhases * B segments in ticket order
  std::vector<int> pcounts;           // items per (image, phase)
  int ptotal = 0;
  int ngroups = 0;
  PersistSegment* d_psegs = nullptr;
  int* d_pcounts = nullptr;
  unsigned* d_ctrl = nullptr;        // ticket, then done[B][kPersistPhases]
  int pgrid = 0;
  cudaGraph_t pgraph = nullptr;
  cudaGraphExec_t pexec = nullptr;
};

namespace {

int bfail(bsf_batch_t b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define BSF_BCUDA(b, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? BSF_ENOMEM : BSF_ECUDA, "%s: %s", \
                   #call, cudaGetErrorString(e_));                                      \
  } while (0)

int height_class(int Hp) { return Hp <= 384 ? 0 : (Hp <= 768 ? 1 : (Hp <= 1536 ? 2 : 3)); }

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

void drop_graph(bsf_batch_t b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (b->pexec) cudaGraphExecDestroy(b->pexec);
  if (b->pgraph) cudaGraphDestroy(b->pgraph);
  b->pexec = nullptr;
  b->pgraph = nullptr;
}

void free_plan(bsf_batch_t b) {
  drop_graph(b);
  if (b->arena) cudaFree(b->arena);
  if (b->d_imgs) cudaFree(b->d_imgs);
  if (b->d_starts) cudaFree(b->d_starts);
  if (b->d_psegs) cudaFree(b->d_psegs);
  if (b->d_pcounts) cudaFree(b->d_pcounts);
  if (b->d_ctrl) cudaFree(b->d_ctrl);
  b->arena = nullptr;
  b->d_imgs = nullptr;
  b->d_starts = nullptr;
  b->d_psegs = nullptr;
  b->d_pcounts = nullptr;
  b->d_ctrl = nullptr;
  b->arena_bytes = 0;
  b->planned = false;
}

std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess)
    return "unknown";
  std::string s = p.name;
  for (char& c : s)
    if (c == ' ') c = '_';
  return s;
}

void load_cache(bsf_batch_t b) {
  if (b->tune_cache.empty()) return;
  FILE* f = std::fopen(b->tune_cache.c_str(), "r");
  if (!f) return;
  char name[256];
  int cls, n, ch;
  const std::string me = gpu_name();
  while (std::fscanf(f, "%255s %d %d %d", name, &cls, &n, &ch) == 4) {
    if (me != name || n != b->n) continue;
    if (cls >= 0 && cls < 4 && ch >= kScanChunkMin) b->tune_chunk[cls] = ch;
    // persistent launch: 100 rows per row item, 101 finite-difference tile rows / 8, 102 blocks per SM
    if (cls == 100 && ch >= 1 && ch <= 64) { b->pshape.rows_per_item = ch; b->tuned_persist = 1; }
    if (cls == 101 && ch >= 1 && ch <= 16) { b->pshape.stencil_rows = ch; b->tuned_persist = 1; }
    if (cls == 102 && ch >= 1 && ch <= 32) { b->ctas_per_sm = ch; b->tuned_persist = 1; }
    if (cls == 103 && ch >= 0 && ch <= 4096) { b->group_mb = ch; b->tuned_persist = 1; }
  }
  std::fclose(f);
}

void save_cache(bsf_batch_t b) {
  if (b->tune_cache.empty()) return;
  FILE* f = std::fopen(b->tune_cache.c_str(), "a");
  if (!f) return;
  const std::string me = gpu_name();
  for (int c = 0; c < 4; ++c)
    if (b->tune_chunk[c]) std::fprintf(f, "%s %d %d %d\n", me.c_str(), c, b->n, b->tune_chunk[c]);
  if (b->tuned_persist) {
    std::fprintf(f, "%s 100 %d %d\n", me.c_str(), b->n, b->pshape.rows_per_item);
    std::fprintf(f, "%s 101 %d %d\n", me.c_str(), b->n, b->pshape.stencil_rows);
    std::fprintf(f, "%s 102 %d %d\n", me.c_str(), b->n, b->ctas_per_sm);
    std::fprintf(f, "%s 103 %d %d\n", me.c_str(), b->n, b->group_mb);
  }
  std::fclose(f);
}

// One image through the per-image kernels (row sums, three vertical
// directions, finite differences) with its own parameters.
int run_one(bsf_batch_t b, const BatchImage& im) {
  cudaError_t e = bsf_launch_scan_rows(BSF_FIX64, b->n, im.img, b->dtype, im.ld, im.H, im.W, im.R, 0,
                                       b->boundary, b->q, im.S, im.pitch, im.Hp, im.Wp, b->st,
                                       b->stream);
  const int skews[3] = {0, 1, -1};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = bsf_launch_vscan(BSF_FIX64, b->n, skews[k], false, im.S, im.pitch, im.Hp, im.Wp, im.ch,
                         im.agg, nullptr, b->stream);
  if (e == cudaSuccess)
    e = bsf_launch_stencil_d1(BSF_FIX64, b->n, im.S, im.pitch, im.R, im.cov, BSF_COV_C, b->step_rule, im.H,
                              im.W, 0, im.H, b->q, im.out, b->out_dtype, im.ldo, b->st, b->stream);
  if (e != cudaSuccess) return bfail(b, BSF_ECUDA, "per-image launch: %s", cudaGetErrorString(e));
  return BSF_OK;
}

int run_batched(bsf_batch_t b) {
  cudaError_t e = bsf_launch_batch_rows(b->n, b->dtype, b->d_imgs, b->d_starts, b->B,
                                        b->totals[kBatchRows], b->boundary, b->q, b->st, b->stream);
  const int skews[3] = {0, 1, -1};
  const int ph[3] = {kBatchV0, kBatchVp, kBatchVm};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = bsf_launch_batch_vscan(b->n, skews[k], b->d_imgs, b->d_starts + ph[k] * (b->B + 1), b->B,
                               b->totals[ph[k]], b->stream);
  if (e == cudaSuccess)
    e = bsf_launch_batch_stencil(b->n, b->out_dtype, b->d_imgs,
                                 b->d_starts + kBatchStencil * (b->B + 1), b->B,
                                 b->totals[kBatchStencil], b->step_rule, b->q, b->st, b->stream);
  if (e != cudaSuccess) return bfail(b, BSF_ECUDA, "batched launch: %s", cudaGetErrorString(e));
  return BSF_OK;
}

int reset_status(bsf_batch_t b) {
  const size_t a = offsetof(DevStatus, clamp_count);
  const size_t z = offsetof(DevStatus, max_absq_bits) + sizeof(unsigned);
  BSF_BCUDA(b, cudaMemsetAsync(reinterpret_cast<char*>(b->st) + a, 0, z - a, b->stream));
  return BSF_OK;
}

bool same_descs(bsf_batch_t b, int B, const bsf_image_desc* d) {
  if (B != b->B) return false;
  for (int i = 0; i < B; ++i) {
    const bsf_image_desc& a = d[i];
    const bsf_image_desc& p = b->descs[i];
    if (a.H != p.H || a.W != p.W || a.img != p.img || a.dtype != p.dtype || a.ld != p.ld ||
        a.cov != p.cov || a.out != p.out || a.out_dtype != p.out_dtype || a.ldo != p.ldo)
      return false;
  }
  return true;
}

// Block offsets of the batched launches and work items of the persistent
// launch, from the images' chunk heights and the persistent item shape;
// uploads them (synchronous) and drops recorded graphs.
int layout(bsf_batch_t b) {
  const int B = b->B;
  b->starts.assign(kBatchPhases * (B + 1), 0);
  for (int p = 0; p < kBatchPhases; ++p) {
    long long acc = 0;
    for (int i = 0; i < B; ++i) {
      b->starts[p * (B + 1) + i] = (int)acc;
      const BatchImage& im = b->imgs[i];
      long long blocks = 0;
      if (p == kBatchRows) {
        blocks = im.Hp;
      } else if (p == kBatchStencil) {
        blocks = (long long)((im.W + 31) / 32) * ((im.H + 7) / 8);
      } else {
        const int Nu = p == kBatchV0 ? im.Wp : im.Wp + im.Hp - 1;
        blocks = (long long)((Nu + 127) / 128) * ((im.Hp + im.ch - 1) / im.ch);
      }
      if (acc + blocks >= (1LL << 31)) return bfail(b, BSF_EINVAL, "batch too large");
      acc += blocks;
    }
    b->starts[p * (B + 1) + B] = (int)acc;
    b->totals[p] = (int)acc;
  }
  // the persistent launch: groups of consecutive images whose running sums
  // fit group_mb, tickets group by group and within a group phase by phase
  b->pcounts.assign((size_t)B * kPersistPhases, 0);
  for (int i = 0; i < B; ++i)
    for (int p = 0; p < kPersistPhases; ++p)
      b->pcounts[i * kPersistPhases + p] = bsf_persistent_items(b->imgs[i], p, b->pshape);
  b->psegs.clear();
  b->ngroups = 0;
  long long ticket = 0;
  const double budget = b->group_mb > 0 ? b->group_mb * 1048576.0 : 1e300;
  for (int g0 = 0; g0 < B;) {
    int g1 = g0 + 1;
    double bytes = (double)b->imgs[g0].pitch * b->imgs[g0].Hp * 8;
    while (g1 < B && bytes + (double)b->imgs[g1].pitch * b->imgs[g1].Hp * 8 <= budget) {
      bytes += (double)b->imgs[g1].pitch * b->imgs[g1].Hp * 8;
      ++g1;
    }
    for (int p = 0; p < kPersistPhases; ++p)
      for (int i = g0; i < g1; ++i) {
        b->psegs.push_back(PersistSegment{(int)ticket, p, i, 0});
        ticket += b->pcounts[i * kPersistPhases + p];
        if (ticket >= (1LL << 31)) return bfail(b, BSF_EINVAL, "batch too large");
      }
    ++b->ngroups;
    g0 = g1;
  }
  b->ptotal = (int)ticket;
  int dev = 0, sms = 0;
  BSF_BCUDA(b, cudaGetDevice(&dev));
  BSF_BCUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int occ = bsf_persistent_occupancy(b->n, b->dtype, b->out_dtype);
  const int per_sm = b->ctas_per_sm > 0 && b->ctas_per_sm < occ ? b->ctas_per_sm : occ;
  b->pgrid = sms * per_sm;
  drop_graph(b);
  BSF_BCUDA(b, cudaMemcpyAsync(b->d_imgs, b->imgs.data(), sizeof(BatchImage) * B, cudaMemcpyHostToDevice,
                               b->stream));
  BSF_BCUDA(b, cudaMemcpyAsync(b->d_starts, b->starts.data(), sizeof(int) * b->starts.size(),
                               cudaMemcpyHostToDevice, b->stream));
  BSF_BCUDA(b, cudaMemcpyAsync(b->d_psegs, b->psegs.data(), sizeof(PersistSegment) * b->psegs.size(),
                               cudaMemcpyHostToDevice, b->stream));
  BSF_BCUDA(b, cudaMemcpyAsync(b->d_pcounts, b->pcounts.data(), sizeof(int) * b->pcounts.size(),
                               cudaMemcpyHostToDevice, b->stream));
  BSF_BCUDA(b, cudaStreamSynchronize(b->stream));
  return BSF_OK;
}

// The persistent launch: zero the ticket and the phase counters, then one
// kernel over every work item of the batch.
int run_persistent(bsf_batch_t b) {
  BSF_BCUDA(b, cudaMemsetAsync(b->d_ctrl, 0, sizeof(unsigned) * (1 + (size_t)b->B * kPersistPhases),
                               b->stream));
  cudaError_t e = bsf_launch_batch_persistent(b->n, b->dtype, b->out_dtype, b->pgrid, b->d_imgs, b->d_psegs,
                                              (int)b->psegs.size(), b->d_pcounts, b->ptotal, b->pshape,
                                              b->boundary, b->q, b->step_rule,
                                              b->d_ctrl, b->d_ctrl + 1, b->wait_limit, b->test_withhold, b->st,
                                              b->stream);
  if (e != cudaSuccess) return bfail(b, BSF_ECUDA, "persistent launch: %s", cudaGetErrorString(e));
  return BSF_OK;
}

// Median-free timing of the persistent launch: the mean of `reps` launches
// after one untimed one.
int time_persistent(bsf_batch_t b, int reps, float* ms) {
  cudaEvent_t e0, e1;
  BSF_BCUDA(b, cudaEventCreate(&e0));
  BSF_BCUDA(b, cudaEventCreate(&e1));
  int rc = reset_status(b);
  if (!rc) rc = run_persistent(b);
  if (!rc) rc = cudaEventRecord(e0, b->stream) == cudaSuccess ? BSF_OK : BSF_ECUDA;
  for (int r = 0; r < reps && !rc; ++r) rc = run_persistent(b);
  if (!rc) rc = cudaEventRecord(e1, b->stream) == cudaSuccess ? BSF_OK : BSF_ECUDA;
  if (!rc) rc = cudaEventSynchronize(e1) == cudaSuccess ? BSF_OK : BSF_ECUDA;
  float t = 0.f;
  if (!rc) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return bfail(b, rc, "timing the persistent launch");
  *ms = t / reps;
  return BSF_OK;
}

// Coordinate descent over the persistent launch's parameters with the batch
// itself as the workload: the scan chunk height of each height class present,
// padded rows per row item, rows of a finite-difference tile (in units of 8)
// and blocks per SM.  Two passes over the parameters; each candidate is kept
// only if it is faster than the best so far.
int tune_persistent(bsf_batch_t b) {
  const int occ = bsf_persistent_occupancy(b->n, b->dtype, b->out_dtype);
  bool present[4] = {false, false, false, false};
  for (const BatchImage& im : b->imgs) present[height_class(im.Hp)] = true;
  float best = 0.f;
  int rc;
  if ((rc = time_persistent(b, 3, &best))) return rc;
  auto try_value = [&](int* slot, int value, bool chunk_class, int cls) -> int {
    const int old = *slot;
    if (value == old) return BSF_OK;
    *slot = value;
    if (chunk_class)
      for (BatchImage& im : b->imgs)
        if (height_class(im.Hp) == cls) im.ch = value;
    int r = layout(b);
    float t = 0.f;
    if (!r) r = time_persistent(b, 3, &t);
    if (r) return r;
    if (t < best) {
      best = t;
      return BSF_OK;
    }
    *slot = old;
    if (chunk_class)
      for (BatchImage& im : b->imgs)
        if (height_class(im.Hp) == cls) im.ch = old;
    return layout(b);
  };
  for (int c = 0; c < 4; ++c)
    if (!b->tune_chunk[c]) b->tune_chunk[c] = kScanChunk;
  if (b->ctas_per_sm <= 0) b->ctas_per_sm = occ;
  for (int pass = 0; pass < 2; ++pass) {
    for (int cls = 0; cls < 4; ++cls) {
      if (!present[cls]) continue;
      for (int ch : {32, 48, 64, 96, 128})
        if ((rc = try_value(&b->tune_chunk[cls], ch, true, cls))) return rc;
    }
    for (int r : {1, 2, 4, 8})
      if ((rc = try_value(&b->pshape.rows_per_item, r, false, 0))) return rc;
    for (int r : {1, 2, 4})
      if ((rc = try_value(&b->pshape.stencil_rows, r, false, 0))) return rc;
    for (int k = 1; k <= occ; ++k)
      if ((rc = try_value(&b->ctas_per_sm, k, false, 0))) return rc;
    for (int mb : {16, 32, 48, 64, 96, 0})
      if ((rc = try_value(&b->group_mb, mb, false, 0))) return rc;
  }
  b->tuned_persist = 1;
  return BSF_OK;
}

}  // namespace

extern "C" {

int bsf_batch_create(bsf_batch_t* out, int n, int boundary) {
  if (!out) return BSF_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 3 || boundary < BSF_ZERO || boundary > BSF_SYMMETRIC) return BSF_EINVAL;
  bsf_batch_t b = new (std::nothrow) bsf_batch();
  if (!b) return BSF_ENOMEM;
  b->n = n;
  b->boundary = boundary;
  if (cudaMalloc(&b->st, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(b->st, 0, sizeof(DevStatus)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    bsf_batch_destroy(b);
    return BSF_ECUDA;
  }
  b->own_stream = true;
  *out = b;
  return BSF_OK;
}

void bsf_batch_destroy(bsf_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_plan(b);
  if (b->st) cudaFree(b->st);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int bsf_batch_set_stream(bsf_batch_t b, void* stream) {
  if (!b) return BSF_EINVAL;
  if (!stream) return bfail(b, BSF_EINVAL, "a batch needs a non-default stream (graph capture)");
  if (b->own_stream) {
    cudaStreamSynchronize(b->stream);
    cudaStreamDestroy(b->stream);
    b->own_stream = false;
  }
  b->stream = (cudaStream_t)stream;
  drop_graph(b);
  return BSF_OK;
}

int bsf_batch_set_precision(bsf_batch_t b, int frac_bits, double value_bound) {
  if (!b) return BSF_EINVAL;
  if (frac_bits < -1 || frac_bits > 62) return bfail(b, BSF_EINVAL, "frac_bits outside [-1, 62]");
  b->frac_req = frac_bits;
  b->has_bound = value_bound > 0.0;
  b->value_bound = value_bound;
  return BSF_OK;
}

int bsf_batch_set_tune_cache(bsf_batch_t b, const char* path) {
  if (!b) return BSF_EINVAL;
  b->tune_cache = path ? path : "";
  load_cache(b);
  return BSF_OK;
}

int bsf_batch_plan(bsf_batch_t b, int B, const bsf_image_desc* descs, int flags) {
  if (!b || B <= 0 || !descs) return BSF_EINVAL;
  for (int i = 0; i < B; ++i) {
    const bsf_image_desc& d = descs[i];
    if (d.H <= 0 || d.W <= 0 || !d.img || !d.cov || !d.out || d.ld < d.W || d.ldo < d.W ||
        d.dtype != descs[0].dtype || d.out_dtype != descs[0].out_dtype ||
        (d.out_dtype != BSF_F32 && d.out_dtype != BSF_F64))
      return bfail(b, BSF_EINVAL, "bad descriptor %d", i);
  }
  if (b->frac_req < 0 && !b->has_bound && descs[0].dtype != BSF_U8)
    return bfail(b, BSF_EINVAL, "automatic q of a float batch needs a value bound");
  BSF_BCUDA(b, cudaStreamSynchronize(b->stream));
  free_plan(b);

  // per-image reach and mass: one unbounded step solve per image
  std::vector<DevStatus> hst(B);
  DevStatus* dst = nullptr;
  ushort4* Lf = nullptr;
  long long maxpx = 0;
  for (int i = 0; i < B; ++i) maxpx = std::max(maxpx, (long long)descs[i].H * descs[i].W);
  BSF_BCUDA(b, cudaMalloc(&dst, sizeof(DevStatus) * B));
  BSF_BCUDA(b, cudaMalloc(&Lf, sizeof(ushort4) * maxpx));
  BSF_BCUDA(b, cudaMemsetAsync(dst, 0, sizeof(DevStatus) * B, b->stream));
  for (int i = 0; i < B; ++i) {
    cudaError_t e = bsf_launch_steps(descs[i].cov, BSF_COV_C, descs[i].H, descs[i].W, b->n,
                                     b->step_rule, BSF_DIRS_CARTESIAN, -1, Lf, dst + i, b->stream);
    if (e != cudaSuccess) { cudaFree(dst); cudaFree(Lf); return bfail(b, BSF_ECUDA, "steps"); }
  }
  BSF_BCUDA(b, cudaMemcpyAsync(hst.data(), dst, sizeof(DevStatus) * B, cudaMemcpyDeviceToHost, b->stream));
  BSF_BCUDA(b, cudaStreamSynchronize(b->stream));
  cudaFree(dst);
  cudaFree(Lf);

  // common q: the smallest image-wise choice, so one max|Q| bound holds for all
  const double vmax = descs[0].dtype == BSF_U8 ? 255.0 : b->value_bound;
  int q = 62;
  for (int i = 0; i < B; ++i) {
    float m;
    std::memcpy(&m, &hst[i].max_mass_bits, sizeof m);
    const double lm = std::log2(std::max(1.0, (double)m));
    const int qi = (int)std::floor(62.0 - std::log2(std::max(vmax, 1e-300)) - lm) - 1;
    q = std::min(q, qi);
  }
  b->q = b->frac_req >= 0 ? b->frac_req : std::max(0, std::min(q, 36));

  // layout
  b->B = B;
  b->dtype = descs[0].dtype;
  b->out_dtype = descs[0].out_dtype;
  b->descs.assign(descs, descs + B);
  b->imgs.resize(B);
  std::vector<size_t> offS(B), offA(B);
  size_t total = 0;
  for (int i = 0; i < B; ++i) {
    BatchImage& im = b->imgs[i];
    const bsf_image_desc& d = descs[i];
    im.img = d.img; im.ld = d.ld; im.cov = d.cov; im.out = d.out; im.ldo = d.ldo;
    im.H = d.H; im.W = d.W;
    im.R = std::max(hst[i].max_reach, 3 * b->n);
    im.Hp = d.H + 2 * im.R;
    im.Wp = d.W + 2 * im.R;
    im.pitch = (im.Wp + 31) / 32 * 32;
    const int cls = height_class(im.Hp);
    im.ch = b->tune_chunk[cls] ? b->tune_chunk[cls] : kScanChunk;
    if ((long long)im.pitch * im.Hp >= (1LL << 31)) return bfail(b, BSF_EINVAL, "image %d too large", i);
    offS[i] = total;
    total += round256((size_t)im.pitch * im.Hp * 8);
    offA[i] = total;
    const size_t nch = (size_t)(im.Hp + kScanChunkMin - 1) / kScanChunkMin;
    total += round256(nch * b->n * (size_t)(im.Wp + im.Hp - 1) * 8);
  }
  BSF_BCUDA(b, cudaMalloc(&b->arena, total));
  b->arena_bytes = total;
  for (int i = 0; i < B; ++i) {
    b->imgs[i].S = (char*)b->arena + offS[i];
    b->imgs[i].agg = (char*)b->arena + offA[i];
  }

  // autotune the scan chunk per height class (the class's largest image)
  if (flags & BSF_BATCH_AUTOTUNE) {
    const int cand[3] = {32, 64, 128};
    cudaEvent_t e0, e1;
    BSF_BCUDA(b, cudaEventCreate(&e0));
    BSF_BCUDA(b, cudaEventCreate(&e1));
    for (int cls = 0; cls < 4; ++cls) {
      int best_i = -1;
      for (int i = 0; i < B; ++i)
        if (height_class(b->imgs[i].Hp) == cls &&
            (best_i < 0 || (long long)b->imgs[i].Hp * b->imgs[i].Wp >
                               (long long)b->imgs[best_i].Hp * b->imgs[best_i].Wp))
          best_i = i;
      if (best_i < 0 || b->tune_chunk[cls]) continue;
      BatchImage im = b->imgs[best_i];
      float best_t = 1e30f;
      int best_ch = kScanChunk;
      for (int c = 0; c < 3; ++c) {
        im.ch = cand[c];
        float tsum = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
          int rc = run_one(b, im);  // fills S (the rows pass) and times nothing yet
          if (rc) return rc;
          cudaEventRecord(e0, b->stream);
          const int skews[3] = {0, 1, -1};
          for (int k = 0; k < 3; ++k)
            bsf_launch_vscan(BSF_FIX64, b->n, skews[k], false, im.S, im.pitch, im.Hp, im.Wp, im.ch,
                             im.agg, nullptr, b->stream);
          cudaEventRecord(e1, b->stream);
          BSF_BCUDA(b, cudaEventSynchronize(e1));
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) tsum += t;
        }
        if (tsum < best_t) { best_t = tsum; best_ch = cand[c]; }
      }
      b->tune_chunk[cls] = best_ch;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < B; ++i) b->imgs[i].ch = b->tune_chunk[height_class(b->imgs[i].Hp)];
    save_cache(b);
  }

  BSF_BCUDA(b, cudaMalloc(&b->d_imgs, sizeof(BatchImage) * B));
  BSF_BCUDA(b, cudaMalloc(&b->d_starts, sizeof(int) * kBatchPhases * (B + 1)));
  BSF_BCUDA(b, cudaMalloc(&b->d_psegs, sizeof(PersistSegment) * kPersistPhases * (size_t)B));
  BSF_BCUDA(b, cudaMalloc(&b->d_pcounts, sizeof(int) * kPersistPhases * (size_t)B));
  BSF_BCUDA(b, cudaMalloc(&b->d_ctrl, sizeof(unsigned) * (1 + (size_t)B * kPersistPhases)));
  int rc = layout(b);
  if (rc) return rc;
  b->planned = true;
  if ((flags & BSF_BATCH_AUTOTUNE) && !b->tuned_persist) {
    if ((rc = tune_persistent(b))) return rc;
    save_cache(b);
  }
  return BSF_OK;
}

int bsf_filter_batched(bsf_batch_t b, int B, const bsf_image_desc* descs, int flags) {
  if (!b || !descs) return BSF_EINVAL;
  if (!b->planned || !same_descs(b, B, descs))
    return bfail(b, BSF_ESTATE, "descriptors differ from the plan (call bsf_batch_plan)");
  int rc;
  if (flags & BSF_BATCH_PERSISTENT) {
    if (flags & BSF_BATCH_GRAPH) {
      if (!b->pexec) {
        BSF_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        rc = reset_status(b);
        if (!rc) rc = run_persistent(b);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return bfail(b, BSF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        b->pgraph = g;
        BSF_BCUDA(b, cudaGraphInstantiate(&b->pexec, b->pgraph, 0));
      }
      BSF_BCUDA(b, cudaGraphLaunch(b->pexec, b->stream));
      return BSF_OK;
    }
    if ((rc = reset_status(b))) return rc;
    return run_persistent(b);
  }
  if (flags & BSF_BATCH_PER_IMAGE) {
    if ((rc = reset_status(b))) return rc;
    for (int i = 0; i < B; ++i)
      if ((rc = run_one(b, b->imgs[i]))) return rc;
    return BSF_OK;
  }
  if (flags & BSF_BATCH_GRAPH) {
    if (!b->exec) {
      BSF_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      rc = reset_status(b);
      if (!rc) rc = run_batched(b);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (rc) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) return bfail(b, BSF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
      b->graph = g;
      BSF_BCUDA(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    BSF_BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
    return BSF_OK;
  }
  if ((rc = reset_status(b))) return rc;
  return run_batched(b);
}

int bsf_batch_status(bsf_batch_t b) {
  if (!b) return BSF_EINVAL;
  BSF_BCUDA(b, cudaMemcpyAsync(&b->host_st, b->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, b->stream));
  BSF_BCUDA(b, cudaStreamSynchronize(b->stream));
  const int err = b->host_st.err;
  BSF_BCUDA(b, cudaMemsetAsync(&b->st->err, 0, sizeof(int), b->stream));
  BSF_BCUDA(b, cudaStreamSynchronize(b->stream));
  return err;
}

int bsf_batch_get_info(bsf_batch_t b, bsf_batch_info_t* info) {
  if (!b || !info) return BSF_EINVAL;
  std::memset(info, 0, sizeof *info);
  info->B = b->B;
  info->frac_bits = b->q;
  info->arena_bytes = (long long)b->arena_bytes;
  for (int c = 0; c < 4; ++c) info->scan_chunk[c] = b->tune_chunk[c] ? b->tune_chunk[c] : kScanChunk;
  for (int p = 0; p < kBatchPhases; ++p) info->blocks[p] = b->totals[p];
  long long px = 0;
  for (const BatchImage& im : b->imgs) px += (long long)im.H * im.W;
  info->pixels = px;
  info->graph_ready = b->exec != nullptr;
  info->persist_items = b->ptotal;
  info->persist_groups = b->ngroups;
  info->persist_grid = b->pgrid;
  info->rows_per_item = b->pshape.rows_per_item;
  info->stencil_tile_rows = 8 * b->pshape.stencil_rows;
  info->persist_graph_ready = b->pexec != nullptr;
  return BSF_OK;
}

int bsf_batch_set_option(bsf_batch_t b, int option, long long value) {
  if (!b) return BSF_EINVAL;
  switch (option) {
    case BSF_BATCH_OPT_WAIT_LIMIT:
      if (value < 1 || value > (1LL << 30)) return bfail(b, BSF_EINVAL, "wait limit outside [1, 2^30]");
      b->wait_limit = (int)value;
      break;
    case BSF_BATCH_OPT_TEST_WITHHOLD:
      b->test_withhold = value != 0;
      break;
    case BSF_BATCH_OPT_ROWS_PER_ITEM:
      if (value < 1 || value > 64) return bfail(b, BSF_EINVAL, "rows per item outside [1, 64]");
      b->pshape.rows_per_item = (int)value;
      b->tuned_persist = 1;
      break;
    case BSF_BATCH_OPT_STENCIL_ROWS:
      if (value != 8 && value != 16 && value != 32 && value != 64)
        return bfail(b, BSF_EINVAL, "finite-difference tile rows must be 8, 16, 32 or 64");
      b->pshape.stencil_rows = (int)value / 8;
      b->tuned_persist = 1;
      break;
    case BSF_BATCH_OPT_GROUP_MB:
      if (value < 0 || value > 4096) return bfail(b, BSF_EINVAL, "group budget outside [0, 4096] MiB");
      b->group_mb = (int)value;
      b->tuned_persist = 1;
      break;
    case BSF_BATCH_OPT_BLOCKS_PER_SM:
      if (value < 0 || value > 32) return bfail(b, BSF_EINVAL, "blocks per SM outside [0, 32]");
      b->ctas_per_sm = (int)value;
      b->tuned_persist = value != 0;
      break;
    default:
      return bfail(b, BSF_EINVAL, "unknown batch option %d", option);
  }
  drop_graph(b);  // the recorded launches carry the old parameters
  if (b->planned && option != BSF_BATCH_OPT_WAIT_LIMIT && option != BSF_BATCH_OPT_TEST_WITHHOLD)
    return layout(b);
  return BSF_OK;
}

void* bsf_batch_stream(bsf_batch_t b) { return b ? (void*)b->stream : nullptr; }

const char* bsf_batch_last_error(bsf_batch_t b) { return b ? b->msg : "NULL batch"; }

}  // extern "C"
