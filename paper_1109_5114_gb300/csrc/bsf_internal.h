// Internal declarations shared by the translation units of libbsf.so.
// Nothing here is part of the public ABI (include/bsf.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bsf.h"

// Device-side status word of a context.  Kernels record the first error code
// and running maxima here; bsf_status() reads and clears it.
struct DevStatus {
  int err;                          // first device-side error (BSF_E*), 0 = none
  unsigned clamp_count;             // pixels whose covariance was clamped to e(phi)
  unsigned bad_count;               // pixels with non-finite covariance
  unsigned range_count;             // pixels whose taps exceeded R (steps reset to 1)
  unsigned overflow_count;          // pixels whose bound max|Q| * mass exceeded the modulus
  int max_reach;                    // largest tap reach of the last step solve
  unsigned max_mass_bits;           // float32 bits of the largest prod L^n (non-negative)
  unsigned max_absq_bits;           // float32 bits of an upper bound of max |Q(f)|
  unsigned long long max_absf_bits; // float64 bits of max |f| (value reduction kernel)
  unsigned max_absg_bits;           // float32 bits of max |gout| (backward)
};

// Default and smallest chunk height (rows per chunk) of the three-phase
// vertical running sums; workspace is sized for the smallest.
constexpr int kScanChunk = 48;
constexpr int kScanChunkMin = 16;

// Launchers; each returns the launch status (cudaGetLastError()).
cudaError_t bsf_launch_steps(const float* cov, int cov_kind, int H, int W, int n, int rule,
                             int dirset, int R, ushort4* Lf, DevStatus* st, cudaStream_t s);

cudaError_t bsf_launch_absmax(const void* img, int dtype, long long ld, int H, int W,
                              DevStatus* st, cudaStream_t s);

// prec: BSF_FIX64 (uint64), BSF_FIX128 (uint128), BSF_F64ACC (float64) or
// BSF_F32KAHAN (double-float) element type of the running sums.
// Row running sums of image rows row0 - R .. row0 - R + Hp - 1 (extended).
cudaError_t bsf_launch_scan_rows(int prec, int n, const void* img, int dtype, long long ld,
                                 int H, int W, int R, int row0, int boundary, int q, void* S,
                                 long long pitch, int Hp, int Wp, DevStatus* st, cudaStream_t s);

// Vertical running sums along d3 (skew 0), d2 (skew +1), d4 (skew -1), in place
// on S.  agg and carry each hold nchunks * n * Nu elements, Nu = Wp + Hp - 1.
cudaError_t bsf_launch_vscan(int prec, int n, int skew, bool reverse, void* S, long long pitch,
                             int Hp, int Wp, int chunk, void* agg, void* carry, cudaStream_t s);

// Single-pass vertical running sums (decoupled look-back).  aggs and incls
// each hold bsf_vscan_lb_bytes() bytes; sync_words holds *sync_bytes (zeroed
// by the launcher).  Waits poll at most spin_limit times.
size_t bsf_vscan_lb_bytes(int elem_bytes, int n, int Hp, int Wp, size_t* sync_bytes);
// Fixed-point types only.  reverse: suffix sums (the transpose).
// test_unpublished != 0 leaves the first chunk's flags unset (failure injection).
cudaError_t bsf_launch_vscan_lb(int prec, int n, int skew, bool reverse, bool short_tiles,
                                void* S, long long pitch, int Hp, int Wp, void* aggs, void* incls,
                                unsigned* sync_words, int spin_limit, int test_unpublished,
                                DevStatus* st, cudaStream_t s);

// In-place n-fold suffix sums along each padded row (transpose of the d1 sum).
cudaError_t bsf_launch_suffix_rows(int elem_bytes, int n, void* S, long long pitch, int Hp, int Wp,
                                   cudaStream_t s);

// Backward of the D1 filter (uint64, or uint128 for contexts with 128-bit
// running sums): max|gout| reduction, tap scatter into G (zeroed by the
// caller), extension fold of G (via Gx: [Hp][W]) into gimg.  elem_bytes (8
// or 16) is the adjoint element width.
cudaError_t bsf_launch_gabsmax(const float* gout, long long ldg, int H, int W, DevStatus* st,
                               cudaStream_t s);
// Scatter of the pixels of rows [row0, row0 + rows) into G (the band's padded
// rows); qg >= 0 fixes the weights' fraction bits, -1 takes them from the
// device maximum of |gout| (bsf_launch_gabsmax).
cudaError_t bsf_launch_scatter_d1(int n, int elem_bytes, void* G, long long pitch, int R, const float* cov,
                                  int cov_kind, int rule, const float* gout, long long ldg, int H,
                                  int W, int row0, int rows, int qg, DevStatus* st, cudaStream_t s,
                                  bool after_absmax = false);
// Band fold: G's Hb padded rows (row 0 = image row row0 - R) folded by the
// extension rule into image rows [a0, a1) as exact sums (acc: elements of
// elem_bytes, two's complement, lda elements per row).
cudaError_t bsf_launch_fold_band(int elem_bytes, const void* G, long long pitch, int Hb, int H, int W, int R,
                                 int row0, int boundary, void* Gx, int a0, int a1, void* acc,
                                 long long lda, cudaStream_t s);
// acc += halo modulo 2^(8 elem_bytes), rows x W.
cudaError_t bsf_launch_add_rows(int elem_bytes, void* acc, long long lda, const void* halo, long long ldh,
                                int rows, int W, cudaStream_t s);
// gimg = RN32(acc) 2^-qg, rows x W.
cudaError_t bsf_launch_grad_finalize(int elem_bytes, const void* acc, long long lda, int rows, int W, int qg,
                                     float* gimg, long long ldo, cudaStream_t s);
// qg = 54 - ceil(log2 m) of the float32 value of m, clamped to [0, 100]
// (64-bit adjoint sums); the 128-bit sums' rule 118 - ceil(log2 m) in [0, 126].
int bsf_grad_q_host(double m);
int bsf_grad_q_host_wide(double m);
cudaError_t bsf_launch_fold(const void* G, long long pitch, int Hp, int H, int W, int R,
                            int boundary, void* Gx, float* gimg, long long ldo, const DevStatus* st,
                            cudaStream_t s);

// ---- batched form: one launch per phase over every image of a batch --------
// Per-image parameters of a batch (device array).  S and agg point into the
// batch's arena; q is common to the batch.
struct BatchImage {
  const void* img;
  long long ld;
  const float* cov;
  void* out;
  long long ldo;
  void* S;
  void* agg;
  long long pitch;
  int H, W, R, Hp, Wp, ch;
};
// Phases with their own block ranges: starts[phase * (B + 1) + i] is the first
// block of image i (starts[... + B] = total blocks).
enum { kBatchRows = 0, kBatchV0 = 1, kBatchVp = 2, kBatchVm = 3, kBatchStencil = 4, kBatchPhases = 5 };

// The persistent batch kernel (bsf_persistent.cu): eight phases of work
// items (rows, three vertical directions in two passes each, finite
// differences).  A segment is the run of tickets of one image's items of one
// phase; segments are sorted by their first ticket.  counts[i * 8 + p] is
// the number of items of image i in phase p, and done holds one counter per
// image and phase (zeroed, as the ticket, before each launch).
constexpr int kPersistPhases = 8;
struct PersistentShape {
  int rows_per_item;  // padded rows of one item of the row phase
  int stencil_rows;   // a finite-difference item is 32 x (8 stencil_rows) pixels
};
struct PersistSegment {
  int first;  // first ticket
  int phase;
  int image;
  int pad;
};
int bsf_persistent_items(const BatchImage& im, int phase, PersistentShape shp);
int bsf_persistent_occupancy(int n, int dtype, int out_dtype);
cudaError_t bsf_launch_batch_persistent(int n, int dtype, int out_dtype, int grid, const BatchImage* imgs,
                                        const PersistSegment* segs, int nseg, const int* counts, int total,
                                        PersistentShape shp,
                                        int boundary, int q, int rule, unsigned* ticket, unsigned* done,
                                        int wait_limit, int test_withhold, DevStatus* st, cudaStream_t s);

cudaError_t bsf_launch_batch_rows(int n, int dtype, const BatchImage* imgs, const int* starts, int B,
                                  int total, int boundary, int q, DevStatus* st, cudaStream_t s);
cudaError_t bsf_launch_batch_vscan(int n, int skew, const BatchImage* imgs, const int* starts, int B,
                                   int total, cudaStream_t s);
cudaError_t bsf_launch_batch_stencil(int n, int out_dtype, const BatchImage* imgs, const int* starts,
                                     int B, int total, int rule, int q, DevStatus* st,
                                     cudaStream_t s);

// Finite differences with the per-pixel step solve fused in (cov: [3][H][W]).
// Output rows row0 .. row0 + rows - 1 of an H x W image (S holds that band).
cudaError_t bsf_launch_stencil_d1(int prec, int n, const void* S, long long pitch, int R,
                                  const float* cov, int cov_kind, int rule, int H, int W, int row0,
                                  int rows, int q, void* out, int out_dtype, long long ldo,
                                  DevStatus* st, cudaStream_t s);
// The same, and with after_scans the kernel just before on the stream is the
// last kernel of these running sums: the stencil then starts as its
// programmatic dependent (the step solve overlaps it; the gathers wait).
cudaError_t bsf_launch_stencil_d1_ex(int prec, int n, const void* S, long long pitch, int R,
                                     const float* cov, int cov_kind, int rule, int H, int W, int row0,
                                     int rows, int q, void* out, int out_dtype, long long ldo,
                                     DevStatus* st, cudaStream_t s, bool after_scans);

// Continuous-step stencil (BSF_STEP_D2, n = 1, 2; BSF_FIX64 / BSF_FIX128).
// mode 0: out only; 1: out and the Jacobian planes jac[c * jac_plane + y * ldj + x]
// (d out / d plane c of cov_kind); 2: gout(p) times the Jacobian into the same
// layout (no out).  Rows row0 .. row0 + rows - 1; S holds that band.
cudaError_t bsf_launch_stencil_d2(int prec, int n, int mode, const void* S, long long pitch, int R,
                                  const float* cov, int cov_kind, int H, int W, int row0, int rows,
                                  int q, void* out, int out_dtype, long long ldo, float* jac,
                                  long long ldj, long long jac_plane, const float* gout,
                                  long long ldg, DevStatus* st, cudaStream_t s);
// Image-gradient adjoint of the continuous-step taps into G (uint128, [Hp][pitch],
// zeroed by the caller), and the 128-bit extension fold into gimg; both take
// qg from the device maximum of |gout| (bsf_launch_gabsmax).
cudaError_t bsf_launch_scatter_d2(int n, void* G, long long pitch, int R, const float* cov,
                                  int cov_kind, const float* gout, long long ldg, int H, int W,
                                  int row0, int rows, int qg, DevStatus* st, cudaStream_t s);
cudaError_t bsf_launch_fold128(const void* G, long long pitch, int Hp, int H, int W, int R,
                               int boundary, void* Gx, float* gimg, long long ldo, const DevStatus* st,
                               cudaStream_t s);
// gcov[c][y][x] = gout[y][x] * jac[c][y][x] (jac planes H * ldj apart; gcov [3][H][W]).
cudaError_t bsf_launch_jacobian_vjp(const float* gout, long long ldg, const float* jac,
                                    long long ldj, float* gcov, int H, int W, cudaStream_t s);

// Stencil of the second direction set (dirset BSF_DIRS_SECOND: S holds its
// running sums) or of the pair (BSF_DIRS_PAIR: S the Cartesian running sums,
// S2 the second set's, same pitch).  prec BSF_FIX64 or BSF_FIX128.
cudaError_t bsf_launch_stencil_sets(int prec, int n, int dirset, const void* S, const void* S2,
                                    long long pitch, int R, const float* cov, int cov_kind, int rule,
                                    int H, int W, int row0, int rows, int q, void* out, int out_dtype,
                                    long long ldo, DevStatus* st, cudaStream_t s);

// Extension + quantisation of the image band onto the padded domain (no
// running sum): S[yp][xp] = Q(f~(xp - R, row0 + yp - R)); records max |Q| and
// overflow like bsf_launch_scan_rows.  Fixed point only.
cudaError_t bsf_launch_extend(int prec, const void* img, int dtype, long long ld, int H, int W, int R,
                              int row0, int boundary, int q, void* S, long long pitch, int Hp, int Wp,
                              DevStatus* st, cudaStream_t s);

// n-fold running sums of the second direction set on S in place (three-phase
// scans): e1 = (2,1) and e4 = (-2,1) on the whole grid, e2 = (1,2) and
// e3 = (-1,2) on each row parity.  agg holds bsf_second_scan_elems elements.
size_t bsf_second_scan_elems(int n, int Hp, int Wp, int chunk);
cudaError_t bsf_launch_scans_second(int prec, int n, void* S, long long pitch, int Hp, int Wp, int chunk,
                                    void* agg, cudaStream_t s);

// Tile-restarted pre-integration fused with the stencil (one launch,
// integer steps, any direction set; the second set and the pair in fixed
// point): bsf_tile_size gives the tile side T (a
// multiple of 32) for this element precision and padding within max_smem
// bytes of shared memory per block, or 0 when no tile of at least 64 fits.
// prec BSF_FIX32/64/128, BSF_F64ACC or BSF_F32KAHAN.  Outputs rows
// [row0, row0 + rows).
// windows: 2 for the pair of direction sets (two windows per block), else 1.
int bsf_tile_size(int prec, int R, int max_smem, int windows);
cudaError_t bsf_launch_tiles(int prec, int n, int dirset, const void* img, int dtype, long long ld, int H, int W,
                             int R, int boundary, int row0, int rows, int TT, int q, const float* cov, int cov_kind,
                             int rule, void* out, int out_dtype, long long ldo, DevStatus* st, cudaStream_t s);

// The sampled continuous box spline (BSF_STEP_SAMPLED): stencil on the
// order-1 running sums S of the direction set (the pair: S Cartesian, S2 the
// second set's).  prec BSF_FIX64 or BSF_FIX128.
cudaError_t bsf_launch_stencil_sampled(int prec, int dirset, const void* S, const void* S2, long long pitch, int R,
                                       const float* cov, int cov_kind, int H, int W, int row0, int rows, int q,
                                       void* out, int out_dtype, long long ldo, DevStatus* st, cudaStream_t s);

// Algorithm 1's split of a field: min over pixels of the condition-2 bound
// (floored at zero) into *min_bits (device, double bits), then the isotropic
// field s2 I and the residual C - s2 I (float32 [3][H][W], BSF_COV_C),
// s2 = RN32(frac * min).
cudaError_t bsf_launch_cov_split(const float* cov, int cov_kind, int H, int W, double frac,
                                 unsigned long long* min_bits, float* iso, float* res,
                                 cudaStream_t s);
