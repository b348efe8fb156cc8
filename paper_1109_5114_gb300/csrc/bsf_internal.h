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
};

// Scan chunk height (rows per chunk) of the vertical running sums.
constexpr int kScanChunk = 64;

// Launchers; each returns the launch status (cudaGetLastError()).
cudaError_t bsf_launch_steps(const float* cov, int cov_kind, int H, int W, int n, int rule,
                             int R, ushort4* Lf, DevStatus* st, cudaStream_t s);

cudaError_t bsf_launch_absmax(const void* img, int dtype, long long ld, int H, int W,
                              DevStatus* st, cudaStream_t s);

cudaError_t bsf_launch_scan_rows(int elem_bytes, int n, const void* img, int dtype, long long ld,
                                 int H, int W, int R, int boundary, int q, void* S,
                                 long long pitch, int Hp, int Wp, DevStatus* st, cudaStream_t s);

// Vertical running sums along d3 (skew 0), d2 (skew +1), d4 (skew -1), in place
// on S.  agg and carry each hold nchunks * n * Nu elements, Nu = Wp + Hp - 1.
cudaError_t bsf_launch_vscan(int elem_bytes, int n, int skew, void* S, long long pitch,
                             int Hp, int Wp, void* agg, void* carry, cudaStream_t s);

cudaError_t bsf_launch_stencil_d1(int elem_bytes, int n, const void* S, long long pitch, int R,
                                  const ushort4* Lf, int H, int W, int q, void* out,
                                  int out_dtype, long long ldo, DevStatus* st, cudaStream_t s);
