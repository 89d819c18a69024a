"""Parity tolerance shared by the GPU tests.

FP32 path vs FP64 oracle, element by element:
    |gpu - oracle| <= rtol * max(|oracle|, floor_frac * mean|oracle|)
with rtol = 1e-5 (the stated FP32 parity bound) and a floor of 1e-3 of the
mean magnitude, so that elements that are nearly zero (a dark texel, a
nearly black shading result) are judged against the scale of their array
rather than against their own tiny value.

Two derived allowances are added where the arithmetic requires them:
  - query/shade: the output's sensitivity to an FP32-sized angular error of
    each light direction (oracle.query_shade_sensitivity), which is far above
    1e-5 only for a rough HDR environment (neighbouring texels differ ~10x);
  - bake depth: 4 ulp of the scene extent, because t* of a Gaussian next to
    the probe cannot be resolved better than the FP32 coordinates it comes
    from;
  - bake outputs: their first-order change under the FP32 rounding of the
    texel direction (2^-24 rad; oracle.bake with_sens), large only where a
    small Gaussian far from the probe decides a texel: turning the ray by
    eps moves its closest point to the centre by t* eps, i.e. t* eps / s in
    units of the Gaussian's scale;
  - surrogate far field: the march's conditioning (oracle.surr_far with
    with_sens), sigma times the FP32 rounding of each cell boundary time,
    summed over the segments.
"""
import numpy as np

RTOL = 1e-5
FLOOR = 1e-3


def excess(gpu, ref, rtol=RTOL, floor=FLOOR, absolute=0.0):
    """Per-element error divided by its allowance (<= 1 passes). `absolute`
    (scalar or per element) adds an allowance derived from the conditioning
    of the element (see the oracle's FP32 sensitivity)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), floor * max(np.mean(np.abs(ref)), 1e-300))
    return np.abs(gpu - ref) / (rtol * scale + absolute)


def assert_close(gpu, ref, rtol=RTOL, floor=FLOOR, what="", absolute=0.0):
    e = excess(gpu, ref, rtol, floor, absolute)
    bad = np.argwhere(e > 1.0)
    if len(bad):
        i = tuple(bad[np.argmax(e[tuple(bad.T)])])
        raise AssertionError(
            f"{what}: {len(bad)} of {e.size} elements outside tolerance (rtol {rtol}); worst at {i}: "
            f"gpu {np.asarray(gpu)[i]!r} oracle {np.asarray(ref)[i]!r} ({e[i]:.2f}x allowance)")
    return float(e.max()) if e.size else 0.0
