// Split-K policy shared by the planner (workspace sizing) and the executor.
//
// A step whose output has few tiles but a long contracted dimension (for
// example the final inner products of two large tensors) would otherwise run
// on a handful of CTAs.  Its K range is then split over several CTAs that
// write FP32 partial products; an ordered reduction adds them.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

namespace tnq {

constexpr int kSplitTargetCtas = 2 * 152;   // aim for two waves of CTAs on the 152 SMs
constexpr double kPartialCapElems = 1 << 26;  // complex64 partial elements (512 MB)

// Skinny steps (few output rows or columns) stay on the CUDA cores even in the
// tensor-core modes: they are bandwidth-bound and a 128-row MMA tile would idle.
// Default rule (the autotuner may override it per step): steps with a small
// side of at most 16 rows are bandwidth-bound and stay on the CUDA cores.
inline bool skinny(int nM, int nN, int nK) {
  (void)nK;
  const int s = nM < nN ? nM : nN;
  return s <= 4;
}

// Whether the rows kernel can run the step (small side <= 32 rows).
inline bool rows_capable(int nM, int nN) { return (nM < nN ? nM : nN) <= 5; }

// Tiny outputs (M, N <= 8) with a long contracted dimension: the dot kernel.
inline bool use_dot(int nM, int nN, int nK) { return nM <= 3 && nN <= 3 && nK >= 10; }

// tiles: CTAs without splitting; kunits: K extent in units the split may cut
// (SIMT: 16-element K slices; tensor cores: 128-byte K blocks); min_units: the
// least K units one split should keep.
inline int split_factor(double tiles, double kunits, double min_units, double out_elems) {
  int s = 1;
  while (tiles * s < kSplitTargetCtas && kunits / (2.0 * s) >= min_units && out_elems * 2.0 * s <= kPartialCapElems)
    s *= 2;
  return s;
}

inline int simt_splits(int nH, int nM, int nN, int nK) {
  double tiles = std::ldexp(1.0, nH) * std::ceil(std::ldexp(1.0, nM) / 64.0) * std::ceil(std::ldexp(1.0, nN) / 64.0);
  return split_factor(tiles, std::ceil(std::ldexp(1.0, nK) / 16.0), 16.0, std::ldexp(1.0, nH + nM + nN));
}

// rows kernel: 128 rows of the large operand per CTA, K staged 32 at a time;
// short K (<= 32) runs unsplit with the row in registers.
inline int rows_splits(int nH, int nM, int nN, int nK) {
  if (nK <= 5) return 1;
  int big = std::max(nM, nN);
  double tiles = std::ldexp(1.0, nH) * std::ceil(std::ldexp(1.0, big) / 128.0);
  return split_factor(tiles, std::ceil(std::ldexp(1.0, nK) / 32.0), 8.0, std::ldexp(1.0, nH + nM + nN));
}

// dot kernel: one CTA per (split, batch entry); each split keeps >= 2048 K elements.
inline int dot_splits(int nH, int nM, int nN, int nK) {
  return split_factor(std::ldexp(1.0, nH), std::ldexp(1.0, nK) / 512.0, 4.0, std::ldexp(1.0, nH + nM + nN));
}

// bf16: 64 complex elements per 128-byte K block of A'; tf32: 16.
inline int tc_splits(int nH, int nM, int nN, int nK, bool bf16) {
  double tiles = std::ldexp(1.0, nH) * std::ceil(std::ldexp(2.0, nM) / 128.0) *
                 std::ceil(std::ldexp(1.0, nN) / 256.0);
  double kblocks = std::ceil(std::ldexp(2.0, nK) / (bf16 ? 64.0 : 32.0));
  return split_factor(tiles, kblocks, 8.0, std::ldexp(1.0, nH + nM + nN));
}

}  // namespace tnq
