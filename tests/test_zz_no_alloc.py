"""nf_loss_noalloc against nf_loss (collected last: the file sorts after the
others, so it runs both alone and after every other test).

The no-alloc entry point keeps its reduction scratch in a file-scope device
array; its loss must equal nf_loss's for the same velocity within the
velocity tolerance (the same kernel and summation order make them equal to
the bit in practice), and two calls in a row must agree (the ticket counter
is cleared at every call).
"""

import numpy as np
import pytest

import nf_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VEL_TOL = 1e-5


def _episode(nf, prec):
    cfg = I.config_chamber(24, steps=2, duct_half_cells=3, cfl_max=1.5)
    ctx = nf.Context(prec, "mgpcg", tol=1e-8, max_iters=2000, cfl_max=cfg["cfl_max"])
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    u0 = [torch.tensor(x, device="cuda") for x in I.gaussian_faces(cfg["grid"], 0.3, 11)]
    ep.set_velocity(u0, project=True)
    ep.step(cfg["steps"])
    return cfg, ctx, ep


@pytest.mark.parametrize("prec,dtype", [("fp64", torch.float64), ("mixed", torch.float32)])
@pytest.mark.parametrize("kind", ["kinetic_energy", "outflow"])
def test_no_alloc_loss_matches_nf_loss_twice_in_a_row(nf, prec, dtype, kind):
    cfg, ctx, ep = _episode(nf, prec)
    J_ref, gU_ref = ep.loss(kind, want_grad=True, dtype=dtype)
    u = ep.velocity(dtype=dtype)
    torch.cuda.synchronize()
    gU = [torch.full_like(t, float("nan")) for t in u]
    J1 = nf.loss_noalloc(kind, cfg["grid"], u, gU=gU)
    J2 = nf.loss_noalloc(kind, cfg["grid"], u)
    ep.close()
    ctx.close()
    assert abs(J1 - J_ref) <= VEL_TOL * abs(J_ref)
    assert J2 == J1
    for a, b in zip(gU, gU_ref):
        np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=VEL_TOL, atol=0)


def test_no_alloc_loss_on_a_side_stream(nf):
    cfg, ctx, ep = _episode(nf, "mixed")
    J_ref = ep.loss("outflow")
    u = ep.velocity(dtype=torch.float32)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        J = nf.loss_noalloc("outflow", cfg["grid"], u)
    ep.close()
    ctx.close()
    assert abs(J - J_ref) <= VEL_TOL * abs(J_ref)


def test_no_alloc_loss_rejects_bad_requests(nf):
    g = I.make_grid(8, 0.01)
    u = [torch.zeros(I.face_shape(g, d), device="cuda") for d in range(3)]
    # too large a grid: refused by the C call before any device work (the
    # binding would refuse these tensors first, so call the ABI directly)
    import ctypes
    from paper_2405_14903_b300 import _lib as L
    from paper_2405_14903_b300.api import grid_struct
    big = grid_struct(dict(g, nx=2048, ny=2048, nz=1024))
    J = ctypes.c_double()
    assert L.lib.nf_loss_noalloc(ctypes.byref(big), L.LOSS["kinetic_energy"],
                                 L.P3(*[t.data_ptr() for t in u]), None, L.NF_F32,
                                 ctypes.byref(J), None) == L.NF_E_INVALID
    assert "too large" in L.lib.nf_last_error(None).decode()
    # outflow without an outlet
    with pytest.raises(nf.NFError, match="outlet"):
        nf.loss_noalloc("outflow", g, u)
    # host arrays are refused by the binding (the C call refuses them too)
    with pytest.raises(TypeError):
        nf.loss_noalloc("kinetic_energy", g, [t.cpu() for t in u])
    # arrays that do not hold the grid's face shapes, or a gradient triple of
    # another shape or dtype, are refused by the binding before the C call
    with pytest.raises(ValueError, match="shape"):
        nf.loss_noalloc("kinetic_energy", dict(g, nx=9), u)
    with pytest.raises(ValueError, match="gU"):
        nf.loss_noalloc("kinetic_energy", g, u, gU=[t.double() for t in u])
    with pytest.raises(ValueError, match="gU"):
        nf.loss_noalloc("kinetic_energy", g, u, gU=[t[:-1].contiguous() for t in u])
    # and a valid call still works afterwards: zero field, zero energy
    assert nf.loss_noalloc("kinetic_energy", g, u) == 0.0
