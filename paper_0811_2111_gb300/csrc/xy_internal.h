// xy_internal.h -- launchers shared between the ABI layer (xy_api.cu) and the
// kernel translation units.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xy.h"
#include "xy_device.cuh"

namespace xyk {

// Arguments of one half-sweep launch over a single lattice.
struct HalfSweepArgs {
  float* theta;          // [2][L][W] split layout, W = L / 2
  int L;
  int W;
  float K;               // beta * J, the factor in exp(K * X), X = -dE / J
  float delta;           // proposal half-window
  xyd::RoundKeys rk;     // Philox round keys of the seed
  uint32_t lattice_id;
  uint32_t sweep;        // Philox counter word 1
  xy_record* rec;        // record of this sweep (zeroed before the red half)
  double beta;           // stored in the record by the black half
};

// Arguments of one fused sweep (both colours and the measure) src -> dst.
struct FusedArgs {
  const float* src;      // [2][L][W] state before the sweep
  float* dst;            // [2][L][W] state after the sweep (distinct buffer)
  int L;
  int W;
  float K;
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id;
  uint32_t sweep;
  xy_record* rec;
  double beta;
};

// Whether the fused kernel handles side L (L a positive multiple of 128).
bool fused_supported(int L);

// One fused sweep; cudaErrorInvalidValue if !fused_supported(a.L).
cudaError_t launch_fused_sweep(int sincos_mode, int reduce_mode, const FusedArgs& a,
                               cudaStream_t stream);

// Unit vectors of n angles with the kernels' sincos of precision `mode`
// (diagnostics and accuracy tests).
cudaError_t launch_eval_unit_vector(int mode, const float* theta, float* c, float* s, int64_t n,
                                    cudaStream_t stream);

// Red (colour 0) then black (colour 1) half-sweep; the black one also adds
// the sweep's bond/spin sums to *rec.  sincos_mode / reduce_mode as in xy.h.
cudaError_t launch_half_sweep(int colour, int sincos_mode, int reduce_mode,
                              const HalfSweepArgs& a, cudaStream_t stream);

// Hot (Philox domain 0) or cold start into the split layout.
cudaError_t launch_start(float* theta, int L, const xyd::RoundKeys& rk, uint32_t lattice_id,
                         int hot, cudaStream_t stream);

// Layout conversions between natural [y][x] order and the split layout.
cudaError_t launch_natural_to_split(const float* nat, float* split, int L, cudaStream_t stream);
cudaError_t launch_split_to_natural(const float* split, float* nat, int L, cudaStream_t stream);

// Philox words for counters (first + i, sweep, lattice_id, domain).
cudaError_t launch_philox_words(const xyd::RoundKeys& rk, uint32_t sweep, uint32_t lattice_id,
                                uint32_t domain, uint32_t first, int64_t n, uint32_t* out,
                                cudaStream_t stream);

// Non-finite check of the split-layout angles: sets *flag to 1 if any is.
cudaError_t launch_check_finite(const float* theta, int64_t n, unsigned int* flag,
                                cudaStream_t stream);

}  // namespace xyk
