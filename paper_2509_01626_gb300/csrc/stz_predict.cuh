// stz_predict.cuh -- interpolation predictors of STZ on the device.
//
// All arithmetic is in the field's precision with single correctly rounded
// operations in a fixed order (op_add / op_sub / op_mul), so compressor and
// decompressor -- and the CPU oracle, which follows the same definitions --
// predict bit for bit the same value.
#pragma once

#include "stz_common.cuh"

namespace stz {

// Eq. 6, the 1D cubic (-1, 9, 9, -1)/16, as mean of the inner pair plus a
// correction: si/2 + (si - so)/16.  A constant is reproduced exactly.
template <typename T>
__device__ __forceinline__ T cubic_1d(T am3, T am1, T ap1, T ap3) {
  T si = op_add(am1, ap1);
  T so = op_add(am3, ap3);
  return op_add(op_mul(si, T(0.5)), op_mul(op_sub(si, so), T(0.0625)));
}

// One-axis boundary rules (Sec. 3.1 opt. 2: boundary points predicted from
// the data available): 0 = midpoint (Eq. 3), 1 = extrapolation from -1 and
// -3, 2 = copy of -1.  Slots of a rule's taps: 0 -> -1, 1 -> +1, 2 -> -3.
enum : int { kMid = 0, kExt = 1, kCopy = 2 };

__device__ __forceinline__ bool rule_uses(int rule, int slot) {
  return slot == 0 || (slot == 1 && rule == kMid) || (slot == 2 && rule == kExt);
}

template <typename T>
__device__ __forceinline__ T apply_rule(int rule, const T w[3]) {
  if (rule == kMid) return op_mul(op_add(w[0], w[1]), T(0.5));
  if (rule == kExt) return op_add(w[0], op_mul(op_sub(w[0], w[2]), T(0.5)));
  return w[0];
}

// coarse-grid offset of a fine tap along an odd axis: -3 -> -1, -1 -> 0,
// +1 -> +1, +3 -> +2; slot form: 0 (-1) -> 0, 1 (+1) -> +1, 2 (-3) -> -1
__device__ __forceinline__ int slot_coarse(int slot) { return slot == 0 ? 0 : (slot == 1 ? 1 : -1); }

// Prediction of the sub-block-K point of the cell at tile index `base` of a
// coarse tile (strides st[3] in elements).  g: the point on G_l, m: G_l
// extent.  Interior: Eq. 6 / Eq. 7 / Eq. 8 by number of odd axes; otherwise
// the separable product of the one-axis rules along the odd axes in the
// order z, y, x (multi-linear Eqs. 3-5 where every rule is the midpoint).
//
// pred selects the ablation of Sec. 3.1: kPredLinear never takes the cubic
// stencils (Eqs. 3-5 everywhere, the one-sided rules at the boundary);
// kPredDirect is Eq. 1, the coarse value of the cell itself (t[base]).
template <int K, typename T, typename I>
__device__ __forceinline__ T level_predict(const T* __restrict__ t, I base, const I st[3],
                                           const int64_t g[3], const int64_t m[3],
                                           int pred = kPredCubic) {
  constexpr int oz = (K >> 2) & 1, oy = (K >> 1) & 1, ox = K & 1;
  constexpr int nodd = oz + oy + ox;
  constexpr int a0 = oz ? 0 : (oy ? 1 : 2);
  constexpr int a1 = nodd >= 2 ? (oz ? (oy ? 1 : 2) : 2) : 2;
  constexpr int a2 = 2;
  const I s0 = st[a0], s1 = st[a1], s2 = st[a2];
  if (pred == kPredDirect) return t[base];
  bool cub = pred == kPredCubic && g[a0] >= 3 && g[a0] + 3 < m[a0];
  if (nodd >= 2) cub = cub && g[a1] >= 3 && g[a1] + 3 < m[a1];
  if (nodd == 3) cub = cub && g[a2] >= 3 && g[a2] + 3 < m[a2];
  if (cub) {
    if (nodd == 1) {
      return cubic_1d(t[base - s0], t[base], t[base + s0], t[base + 2 * s0]);
    } else if (nodd == 2) {
      T si = op_add(op_add(t[base], t[base + s1]), op_add(t[base + s0], t[base + s0 + s1]));
      T so = op_add(op_add(t[base - s0 - s1], t[base - s0 + 2 * s1]),
                    op_add(t[base + 2 * s0 - s1], t[base + 2 * s0 + 2 * s1]));
      return op_add(op_mul(si, T(0.25)), op_mul(op_sub(si, so), T(0.03125)));
    } else {
      const I z = s0, y = s1, x = s2;
      T si = op_add(op_add(op_add(t[base], t[base + x]), op_add(t[base + y], t[base + y + x])),
                    op_add(op_add(t[base + z], t[base + z + x]),
                           op_add(t[base + z + y], t[base + z + y + x])));
      const I zm = -z, zp = 2 * z, ym = -y, yp = 2 * y, xm = -x, xp = 2 * x;
      T so = op_add(op_add(op_add(t[base + zm + ym + xm], t[base + zm + ym + xp]),
                           op_add(t[base + zm + yp + xm], t[base + zm + yp + xp])),
                    op_add(op_add(t[base + zp + ym + xm], t[base + zp + ym + xp]),
                           op_add(t[base + zp + yp + xm], t[base + zp + yp + xp])));
      return op_add(op_mul(si, T(0.125)), op_mul(op_sub(si, so), T(0.015625)));
    }
  }
  int r[3];
  const int ax[3] = {a0, a1, a2};
  for (int i = 0; i < nodd; i++) {
    int a = ax[i];
    r[i] = (g[a] + 1 < m[a]) ? kMid : ((g[a] >= 3) ? kExt : kCopy);
  }
  if (nodd == 1) {
    T w[3] = {T(0), T(0), T(0)};
    for (int q0 = 0; q0 < 3; q0++)
      if (rule_uses(r[0], q0)) w[q0] = t[base + slot_coarse(q0) * s0];
    return apply_rule(r[0], w);
  }
  if (nodd == 2) {
    T w1[3] = {T(0), T(0), T(0)};
    for (int q1 = 0; q1 < 3; q1++) {
      if (!rule_uses(r[1], q1)) continue;
      T w0[3] = {T(0), T(0), T(0)};
      for (int q0 = 0; q0 < 3; q0++)
        if (rule_uses(r[0], q0)) w0[q0] = t[base + slot_coarse(q0) * s0 + slot_coarse(q1) * s1];
      w1[q1] = apply_rule(r[0], w0);
    }
    return apply_rule(r[1], w1);
  }
  T w2[3] = {T(0), T(0), T(0)};
  for (int q2 = 0; q2 < 3; q2++) {
    if (!rule_uses(r[2], q2)) continue;
    T w1[3] = {T(0), T(0), T(0)};
    for (int q1 = 0; q1 < 3; q1++) {
      if (!rule_uses(r[1], q1)) continue;
      T w0[3] = {T(0), T(0), T(0)};
      for (int q0 = 0; q0 < 3; q0++)
        if (rule_uses(r[0], q0))
          w0[q0] = t[base + slot_coarse(q0) * s0 + slot_coarse(q1) * s1 + slot_coarse(q2) * s2];
      w1[q1] = apply_rule(r[0], w0);
    }
    w2[q2] = apply_rule(r[1], w1);
  }
  return apply_rule(r[2], w2);
}

// Base coder (level 1, SZ3-style 1D interpolation): point at index `idx` of
// the level-1 grid, coordinate c along the pass axis (grid stride `st`
// elements per unit), pass stride t, extent m along the axis.  Cubic when
// -3t..+3t fit, else midpoint, else extrapolation, else copy.  I is the index
// type (int for a grid held in shared memory).
template <typename T, typename I>
__device__ __forceinline__ T base_predict(const T* __restrict__ g1, I idx, I st, I c, I t, I m) {
  const I d = t * st;
  T vm1 = g1[idx - d];
  bool p1 = c + t < m, m3 = c - 3 * t >= 0, p3 = c + 3 * t < m;
  if (m3 && p3) return cubic_1d(g1[idx - 3 * d], vm1, g1[idx + d], g1[idx + 3 * d]);
  if (p1) return op_mul(op_add(vm1, g1[idx + d]), T(0.5));
  if (m3) return op_add(vm1, op_mul(op_sub(vm1, g1[idx - 3 * d]), T(0.5)));
  return vm1;
}

}  // namespace stz
