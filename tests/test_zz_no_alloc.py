"""The allocation-free norm entry point against dirac_observables.

dirac_norms_noalloc exists for callers that cannot allocate device memory where they
need a norm (device memory owned by another allocator or a fixed arena, loops that cannot
take cudaMalloc's implicit synchronisation). This file is collected last so that a failure here comes
after every other test has run; it also passes alone in a fresh process."""
import numpy as np
import pytest

import paper_1909_02894_gb300 as D
from paper_1909_02894_gb300 import workloads as W


def test_no_alloc_rejects_grids_beyond_its_static_scratch():
    D.build()
    L = D.lib()
    assert L.dirac_norms_noalloc(None, None, 64, 64, 1.0, 1.0, None, None) == D.DIRAC_EINVAL
    # 8192 x 64 is beyond the 4096-point limit; rejected before any device access
    assert L.dirac_norms_noalloc(1, None, 8192, 64, 1.0, 1.0, 1, None) == D.DIRAC_EINVAL
    assert "4096" in D.dirac_last_error(None)


@pytest.mark.gpu
def test_no_alloc_norms_match_observables_twice():
    torch = pytest.importorskip("torch")
    D.build()
    w = W.graphene_strained(n=256, steps=20)
    with D.Simulation(w, precision=D.DIRAC_C128) as s:
        s.set_state(w.psi0)
        s.step(20, w.dt)
        ref = s.observables()
        psi = torch.empty((2, w.ny, w.nx), dtype=torch.complex128, device="cuda")
        D.dirac_get_state(s.ctx, psi)
        D.dirac_synchronize(s.ctx)
    weight = torch.from_numpy(np.sqrt(w.g11 * w.g22 / w.g00)).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    for call in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        D.dirac_norms_noalloc(psi, weight, w.ax, w.ay, out, stream=stream.cuda_stream)
        stream.synchronize()
        norm, norm_gamma = out.cpu().numpy()
        assert abs(norm - ref["norm"]) <= 1e-12 * ref["norm"], call
        assert abs(norm_gamma - ref["norm_gamma"]) <= 1e-12 * ref["norm_gamma"], call
    # without a weight both entries are the plain norm
    D.dirac_norms_noalloc(psi, None, w.ax, w.ay, out, stream=stream.cuda_stream)
    stream.synchronize()
    n0, n1 = out.cpu().numpy()
    assert abs(n0 - ref["norm"]) <= 1e-12 * ref["norm"] and n0 == n1


def test_no_alloc_binding_refuses_misshaped_tensors_before_any_launch():
    """Shape, dtype and device checks raise ValueError on the host (CPU tensors here,
    so nothing could have been launched)."""
    torch = pytest.importorskip("torch")
    psi = torch.zeros((2, 16, 32), dtype=torch.complex128)
    out = torch.zeros(2, dtype=torch.float64)
    bad = [
        (torch.zeros((16, 32), dtype=torch.complex128), None, out, "shape"),
        (torch.zeros((3, 16, 32), dtype=torch.complex128), None, out, "shape"),
        (psi, torch.zeros((16, 16), dtype=torch.float64), out, "weight"),
        (psi, None, torch.zeros(1, dtype=torch.float64), "out"),
        (psi.to(torch.complex64), None, out, "complex128"),
        (psi, None, out, "CUDA"),
    ]
    for p, w, o, word in bad:
        with pytest.raises(ValueError, match=word):
            D.dirac_norms_noalloc(p, w, 1.0, 1.0, o)
