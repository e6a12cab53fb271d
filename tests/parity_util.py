"""Shared parity measures of the GPU tests.

rel-L2 over the whole grid can hide a localised error in the absorbing layer, where the
state carries little amplitude, so every parity check also bounds the element-wise error
on the layer points (the outer `width` points of each axis and the inner edge,
L* <= |x| <= L of Sec. 3) against the largest oracle amplitude.
"""
import numpy as np

from paper_1909_02894_gb300 import workloads as W


def layer_mask(w):
    """[ny][nx] boolean mask of the absorbing-layer points of workload w."""
    mx = np.zeros(w.nx, dtype=bool)
    my = np.zeros(w.ny, dtype=bool)
    if w.pml_width_x > 0:
        mx[:w.pml_width_x + 1] = True
        mx[w.nx - w.pml_width_x:] = True
    if w.pml_width_y > 0:
        my[:w.pml_width_y + 1] = True
        my[w.ny - w.pml_width_y:] = True
    return mx[None, :] | my[:, None]


def layer_max_rel(got, ref, w):
    """max over layer points of |got - ref| (both components) / max |ref| over all points;
    0 when the workload has no layer."""
    m = layer_mask(w)
    if not m.any():
        return 0.0
    scale = np.abs(ref).max()
    return float(np.abs(got - ref)[:, m].max() / scale)


def assert_parity(got, ref, w, tol):
    """rel-L2 <= tol over all points and the layer's element-wise error <= tol."""
    rel = W.rel_l2(got, ref)
    lay = layer_max_rel(got, ref, w)
    assert rel <= tol and lay <= tol, {"rel_l2": rel, "layer_max_rel": lay, "tol": tol}
    return rel, lay
