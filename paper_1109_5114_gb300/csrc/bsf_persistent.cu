// The whole filter of a batch of images in one persistent launch: a grid of
// resident blocks takes work items from one ticket counter until the batch is
// done.  The items are the passes of the filter (Section 1.1's running sums
// along d1, d3, d2, d4, then the finite differences) cut into pieces:
//
//   phase 0  rows of the padded image: extension + quantisation + d1 sums
//   phase 1  d3 reduction (256 lines x one chunk of rows)
//   phase 2  d3 rescan with the carries folded in
//   phase 3  d2 reduction        phase 4  d2 rescan
//   phase 5  d4 reduction        phase 6  d4 rescan
//   phase 7  finite differences of a tile of 32 x (8 stencil_rows) pixels
//
// The images are cut into groups (consecutive images whose running sums fit
// a byte budget, e.g. a share of the 126 MB L2), and tickets are ordered
// group by group, within a group phase by phase (all of the group's phase p
// before its phase p + 1): a group's running sums are written, scanned and
// read while they are still in L2.  An item of phase p of image i waits until
// every item of phase p - 1 of image i has finished (one counter per image
// and phase).  So a block waits only on items with smaller tickets, which
// blocks that are already running hold: every wait ends, and no phase
// boundary drains the GPU (the next phase, or the next group, starts while
// the last items of a phase finish).
//
// Memory ordering: a finished item's block synchronises, then one thread
// releases (fence at gpu scope) and adds one to the counter; a waiting
// block's thread 0 reads the counter with acquire semantics, the block
// synchronises, and every thread fences before it reads.  The scans read and
// write through L2 (no L1 line of the running sums is filled before the
// finite differences, which read through L1 once an image's sums are final).
//
// Every wait is bounded: after wait_limit polls the block records
// BSF_ETIMEOUT in the status word and goes on (the batch's result is then
// invalid and reported, never hung).  test_withhold != 0 leaves image 0's
// row phase unsignalled (failure injection for tests).
#include "bsf_scan_bodies.cuh"
#include "bsf_stencil.cuh"

namespace {

constexpr int kPThreads = 256;
constexpr int kPLines = 256;  // lines per item of the vertical phases

// the segment (a run of tickets of one image and phase) holding ticket t:
// segments are sorted by their first ticket
__device__ __forceinline__ int p_find(const PersistSegment* __restrict__ segs, int nseg, int t) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].first <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned p_load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int NF, int SKEW, bool APPLY>
__device__ __forceinline__ void p_vscan(const BatchImage& im, int local) {
  const int Nu = SKEW == 0 ? im.Wp : im.Wp + im.Hp - 1;
  const int umin = SKEW == 1 ? -(im.Hp - 1) : 0;
  const int gx = (Nu + kPLines - 1) / kPLines;
  const int bx = local % gx, c = local / gx;
  // the bodies index lines as bx' 128 + threadIdx.x: 256 threads take 2 strips
  if (APPLY)
    vscan_apply_body<uint64_t, NF, SKEW, false, BsfLoadCoherent>((uint64_t*)im.S, im.pitch, im.Hp, im.Wp,
                                                                 umin, Nu, im.ch, (const uint64_t*)im.agg,
                                                                 2 * bx, c);
  else
    vscan_agg_body<uint64_t, NF, SKEW, false, BsfLoadCoherent>((const uint64_t*)im.S, im.pitch, im.Hp,
                                                               im.Wp, umin, Nu, im.ch, (uint64_t*)im.agg,
                                                               2 * bx, c);
}

// resident blocks per SM asked of the register allocator (the finite
// differences set the need: as their own kernel)
template <int NF> struct PersistOcc {
  static constexpr int value = NF == 3 ? 2 : 4;
};

template <int NF, typename In, typename Out>
__global__ void __launch_bounds__(kPThreads, PersistOcc<NF>::value)
k_batch_persistent(const BatchImage* __restrict__ imgs, const PersistSegment* __restrict__ segs, int nseg,
                   const int* __restrict__ counts, int total, PersistentShape shp, int boundary, int q,
                   int rule, float scale_f, double scale_d, unsigned* __restrict__ ticket,
                   unsigned* __restrict__ done, int wait_limit, int test_withhold, DevStatus* st) {
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int t = s_item;
    if (t >= total) return;  // uniform: every thread read the same ticket
    const PersistSegment sg = segs[p_find(segs, nseg, t)];
    const int p = sg.phase, i = sg.image;
    const int local = t - sg.first;
    const BatchImage& im = imgs[i];
    if (p > 0) {
      if (tid == 0) {
        const unsigned need = (unsigned)counts[i * kPersistPhases + (p - 1)];
        const unsigned* cnt = done + i * kPersistPhases + (p - 1);
        int polls = 0;
        while (p_load_acquire(cnt) < need) {
          if (++polls > wait_limit) {
            bsf_set_error(st, BSF_ETIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    if (p == 0) {
      const int y0 = local * shp.rows_per_item, y1 = min(y0 + shp.rows_per_item, im.Hp);
      for (int y = y0; y < y1; ++y)
        scan_rows_body<uint64_t, NF, In, 4>((const In*)im.img, im.ld, im.H, im.W, im.R, 0, boundary,
                                            bsf_pow2_f32(q), q, (uint64_t*)im.S, im.pitch, im.Hp, im.Wp,
                                            st, y);
    } else if (p == 1) {
      p_vscan<NF, 0, false>(im, local);
    } else if (p == 2) {
      p_vscan<NF, 0, true>(im, local);
    } else if (p == 3) {
      p_vscan<NF, 1, false>(im, local);
    } else if (p == 4) {
      p_vscan<NF, 1, true>(im, local);
    } else if (p == 5) {
      p_vscan<NF, -1, false>(im, local);
    } else if (p == 6) {
      p_vscan<NF, -1, true>(im, local);
    } else {
      const int gx = (im.W + 31) / 32;
      const int bx = local % gx, by0 = (local / gx) * shp.stencil_rows;
      for (int j = 0; j < shp.stencil_rows; ++j)
        stencil_d1_body<uint64_t, NF, Out, BSF_DIRS_CARTESIAN, 2>(
            (const uint64_t*)im.S, nullptr, im.pitch, im.R, im.cov, BSF_COV_C, rule, im.H, im.W, 0, im.H,
            scale_f, scale_d, (Out*)im.out, im.ldo, st, bx, by0 + j, tid & 31, tid >> 5, kPThreads / 32);
    }
    __syncthreads();  // the item's writes, and every read of s_item, are done
    if (tid == 0 && !(test_withhold && p == 0 && i == 0)) {
      __threadfence();
      atomicAdd(done + i * kPersistPhases + p, 1u);
    }
  }
}

template <int NF, typename In>
cudaError_t launch_in(int out_dtype, int grid, const BatchImage* imgs, const PersistSegment* segs,
                      int nseg, const int* counts, int total, PersistentShape shp, int boundary, int q, int rule,
                      unsigned* ticket, unsigned* done, int wait_limit, int test_withhold, DevStatus* st,
                      cudaStream_t s) {
  const float sf = ldexpf(1.f, -q);
  const double sd = ldexp(1.0, -q);
  if (out_dtype == BSF_F32)
    k_batch_persistent<NF, In, float><<<grid, kPThreads, 0, s>>>(imgs, segs, nseg, counts, total, shp, boundary,
                                                                 q, rule, sf, sd, ticket, done, wait_limit,
                                                                 test_withhold, st);
  else if (out_dtype == BSF_F64)
    k_batch_persistent<NF, In, double><<<grid, kPThreads, 0, s>>>(imgs, segs, nseg, counts, total, shp,
                                                                  boundary, q, rule, sf, sd, ticket, done,
                                                                  wait_limit, test_withhold, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int NF>
cudaError_t launch_nf(int dtype, int out_dtype, int grid, const BatchImage* imgs, const PersistSegment* segs,
                      int nseg, const int* counts, int total, PersistentShape shp, int boundary, int q, int rule,
                      unsigned* ticket, unsigned* done, int wait_limit, int test_withhold, DevStatus* st,
                      cudaStream_t s) {
  if (dtype == BSF_F32)
    return launch_in<NF, float>(out_dtype, grid, imgs, segs, nseg, counts, total, shp, boundary, q, rule, ticket,
                                done, wait_limit, test_withhold, st, s);
  if (dtype == BSF_U8)
    return launch_in<NF, uint8_t>(out_dtype, grid, imgs, segs, nseg, counts, total, shp, boundary, q, rule,
                                  ticket, done, wait_limit, test_withhold, st, s);
  if (dtype == BSF_F64)
    return launch_in<NF, double>(out_dtype, grid, imgs, segs, nseg, counts, total, shp, boundary, q, rule,
                                 ticket, done, wait_limit, test_withhold, st, s);
  return cudaErrorInvalidValue;
}

template <int NF, typename In, typename Out>
int occupancy_of() {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_batch_persistent<NF, In, Out>, kPThreads, 0) !=
      cudaSuccess)
    return 1;
  return blocks > 0 ? blocks : 1;
}

}  // namespace

int bsf_persistent_items(const BatchImage& im, int phase, PersistentShape shp) {
  if (phase == 0) return (im.Hp + shp.rows_per_item - 1) / shp.rows_per_item;
  if (phase == kPersistPhases - 1) {
    const int tile_rows = 8 * shp.stencil_rows;
    return ((im.W + 31) / 32) * ((im.H + tile_rows - 1) / tile_rows);
  }
  const int skew = phase <= 2 ? 0 : 1;  // d3: Wp lines; d2, d4: Wp + Hp - 1
  const int Nu = skew == 0 ? im.Wp : im.Wp + im.Hp - 1;
  return ((Nu + kPLines - 1) / kPLines) * ((im.Hp + im.ch - 1) / im.ch);
}

int bsf_persistent_occupancy(int n, int dtype, int out_dtype) {
#define BSF_PO(NF)                                                                             \
  if (dtype == BSF_U8) return out_dtype == BSF_F64 ? occupancy_of<NF, uint8_t, double>() : occupancy_of<NF, uint8_t, float>(); \
  if (dtype == BSF_F64) return out_dtype == BSF_F64 ? occupancy_of<NF, double, double>() : occupancy_of<NF, double, float>(); \
  return out_dtype == BSF_F64 ? occupancy_of<NF, float, double>() : occupancy_of<NF, float, float>()
  if (n == 1) { BSF_PO(1); }
  if (n == 2) { BSF_PO(2); }
  BSF_PO(3);
#undef BSF_PO
}

cudaError_t bsf_launch_batch_persistent(int n, int dtype, int out_dtype, int grid, const BatchImage* imgs,
                                        const PersistSegment* segs, int nseg, const int* counts, int total,
                                        PersistentShape shp,
                                        int boundary, int q, int rule, unsigned* ticket, unsigned* done,
                                        int wait_limit, int test_withhold, DevStatus* st, cudaStream_t s) {
  if (n == 1)
    return launch_nf<1>(dtype, out_dtype, grid, imgs, segs, nseg, counts, total, shp, boundary, q, rule, ticket,
                        done, wait_limit, test_withhold, st, s);
  if (n == 2)
    return launch_nf<2>(dtype, out_dtype, grid, imgs, segs, nseg, counts, total, shp, boundary, q, rule, ticket,
                        done, wait_limit, test_withhold, st, s);
  if (n == 3)
    return launch_nf<3>(dtype, out_dtype, grid, imgs, segs, nseg, counts, total, shp, boundary, q, rule, ticket,
                        done, wait_limit, test_withhold, st, s);
  return cudaErrorInvalidValue;
}
