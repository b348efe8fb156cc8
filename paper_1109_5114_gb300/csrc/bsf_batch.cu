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
// The autotuner picks the scan chunk height per size class of the padded
// image (height classes up to 384, 768, 1536 rows and above) by timing the
// vertical running sums of the class's largest image with each candidate;
// the choices can be kept in a text cache file between runs.
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
}

void free_plan(bsf_batch_t b) {
  drop_graph(b);
  if (b->arena) cudaFree(b->arena);
  if (b->d_imgs) cudaFree(b->d_imgs);
  if (b->d_starts) cudaFree(b->d_starts);
  b->arena = nullptr;
  b->d_imgs = nullptr;
  b->d_starts = nullptr;
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
  while (std::fscanf(f, "%255s %d %d %d", name, &cls, &n, &ch) == 4)
    if (me == name && n == b->n && cls >= 0 && cls < 4 && ch >= kScanChunkMin) b->tune_chunk[cls] = ch;
  std::fclose(f);
}

void save_cache(bsf_batch_t b) {
  if (b->tune_cache.empty()) return;
  FILE* f = std::fopen(b->tune_cache.c_str(), "a");
  if (!f) return;
  const std::string me = gpu_name();
  for (int c = 0; c < 4; ++c)
    if (b->tune_chunk[c]) std::fprintf(f, "%s %d %d %d\n", me.c_str(), c, b->n, b->tune_chunk[c]);
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

  // block offsets per phase
  b->starts.assign(kBatchPhases * (B + 1), 0);
  for (int p = 0; p < kBatchPhases; ++p) {
    int acc = 0;
    for (int i = 0; i < B; ++i) {
      b->starts[p * (B + 1) + i] = acc;
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
      acc += (int)blocks;
    }
    b->starts[p * (B + 1) + B] = acc;
    b->totals[p] = acc;
  }
  BSF_BCUDA(b, cudaMalloc(&b->d_imgs, sizeof(BatchImage) * B));
  BSF_BCUDA(b, cudaMalloc(&b->d_starts, sizeof(int) * b->starts.size()));
  BSF_BCUDA(b, cudaMemcpyAsync(b->d_imgs, b->imgs.data(), sizeof(BatchImage) * B,
                               cudaMemcpyHostToDevice, b->stream));
  BSF_BCUDA(b, cudaMemcpyAsync(b->d_starts, b->starts.data(), sizeof(int) * b->starts.size(),
                               cudaMemcpyHostToDevice, b->stream));
  BSF_BCUDA(b, cudaStreamSynchronize(b->stream));
  b->planned = true;
  return BSF_OK;
}

int bsf_filter_batched(bsf_batch_t b, int B, const bsf_image_desc* descs, int flags) {
  if (!b || !descs) return BSF_EINVAL;
  if (!b->planned || !same_descs(b, B, descs))
    return bfail(b, BSF_ESTATE, "descriptors differ from the plan (call bsf_batch_plan)");
  int rc;
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
  return BSF_OK;
}

void* bsf_batch_stream(bsf_batch_t b) { return b ? (void*)b->stream : nullptr; }

const char* bsf_batch_last_error(bsf_batch_t b) { return b ? b->msg : "NULL batch"; }

}  // extern "C"
