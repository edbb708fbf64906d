"""Pins of the oracle's cut-cell Poisson system and projection (no GPU)."""

import numpy as np
import pytest

import nf_inputs as I
from oracle import Grid, mac, project, rasterize


def _system(cfg, t=0.0):
    g = Grid(cfg["grid"])
    alpha = rasterize.fractions(g, cfg["scene"], t)
    us = rasterize.face_solid_velocity(g, cfg["scene"], t)
    return g, project.ProjectionSystem(g, alpha, us)


def _dense(sys_):
    act = np.flatnonzero(sys_.active.ravel())
    n = sys_.active.size
    A = np.zeros((len(act), len(act)))
    for col, cell in enumerate(act):
        e = np.zeros(n)
        e[cell] = 1.0
        A[:, col] = sys_.A(e.reshape(sys_.active.shape)).ravel()[act]
    return A, act


CASES = {
    "sphere8": lambda: I.config_sphere(8),
    "plate8": lambda: I.config_plate(8),
    "chamber8": lambda: I.config_chamber(8, duct_half_cells=2),
    "spheres8": lambda: I.config_spheres(8, count=6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_matrix_symmetric_psd_with_expected_null_space(name):
    g, sys_ = _system(CASES[name]())
    A, act = _dense(sys_)
    assert np.max(np.abs(A - A.T)) <= 1e-15 * np.max(np.abs(A))
    ev = np.linalg.eigvalsh(A)
    assert ev[0] >= -1e-12 * ev[-1]
    nfloat = sum(1 for v in sys_.grounded.values() if not v)
    null = int(np.sum(ev < 1e-10 * ev[-1]))
    assert null == nfloat
    # pinning one cell per floating component makes it positive definite
    lab = sys_.labels.ravel()[act]
    keep = np.ones(len(act), dtype=bool)
    for lab_id, gr in sys_.grounded.items():
        if not gr:
            keep[np.flatnonzero(lab == lab_id)[0]] = False
    np.linalg.cholesky(A[np.ix_(keep, keep)])


def test_outlet_makes_the_chamber_system_nonsingular():
    g, sys_ = _system(CASES["chamber8"]())
    assert all(sys_.grounded.values())
    ev = np.linalg.eigvalsh(_dense(sys_)[0])
    assert ev[0] > 1e-8 * ev[-1]


@pytest.mark.parametrize("name", list(CASES))
def test_cg_matches_dense_direct_solve(name):
    cfg = CASES[name]()
    g, sys_ = _system(cfg)
    Uh = I.gaussian_faces(cfg["grid"], 1.0, 11)
    b = sys_.rhs(Uh)
    P, it, rel = sys_.solve(b, 1e-13)
    A, act = _dense(sys_)
    bb = project.remove_floating_means(b, sys_.labels, sys_.grounded).ravel()[act]
    ref, *_ = np.linalg.lstsq(A, bb, rcond=None)    # minimum-norm solution
    ref_full = np.zeros(sys_.active.size)
    ref_full[act] = ref
    ref_full = project.remove_floating_means(ref_full.reshape(sys_.active.shape),
                                             sys_.labels, sys_.grounded)
    err = np.linalg.norm(P - ref_full) / np.linalg.norm(ref_full)
    assert err < 1e-10


@pytest.mark.parametrize("name", ["sphere16", "plate16", "chamber16"])
def test_divergence_after_projection(name):
    cfg = {"sphere16": lambda: I.config_sphere(16), "plate16": lambda: I.config_plate(16),
           "chamber16": lambda: I.config_chamber(16, duct_half_cells=2)}[name]()
    g, sys_ = _system(cfg, 0.05)
    Uh = I.gaussian_faces(cfg["grid"], 1.0, 12)
    U, P, info = project.project(g, sys_.alpha, sys_.us, Uh, 1e-13)
    div = mac.grad_T(g, U)
    assert np.max(np.abs(div[sys_.active])) <= 1e-10
    # solid faces carry the solid velocity, fluid faces the corrected one
    for d in range(3):
        solid = sys_.alpha[d] == 0.0
        np.testing.assert_array_equal(U[d][solid], sys_.us[d][solid])


def test_fluid_at_rest_with_static_solids_stays_at_rest():
    cfg = I.config_spheres(12, count=5)
    g, sys_ = _system(cfg)
    zero = g.zeros_faces()
    U, P, info = project.project(g, sys_.alpha, sys_.us, zero, 1e-12)
    assert all(np.all(u == 0.0) for u in U) and np.all(P == 0.0)


def test_literal_update_is_idempotent_and_agrees_with_blend_on_full_faces():
    # The printed update U^ - c G P is an alpha-weighted projection: applying
    # it twice changes nothing. The blended update equals it where alpha = 1
    # and equals u_s where alpha = 0.
    cfg = I.config_plate(12)
    g, sys_ = _system(cfg, 0.03)
    Uh = I.gaussian_faces(cfg["grid"], 1.0, 13)
    U1, _, _ = project.project(g, sys_.alpha, sys_.us, Uh, 1e-13, velocity_rule="literal")
    U2, _, _ = project.project(g, sys_.alpha, sys_.us, U1, 1e-13, velocity_rule="literal")
    scale = max(np.abs(u).max() for u in U1)
    assert max(np.abs(a - b).max() for a, b in zip(U1, U2)) < 1e-9 * scale
    Ub, _, _ = project.project(g, sys_.alpha, sys_.us, Uh, 1e-13)
    for d in range(3):
        full = sys_.alpha[d] == 1.0
        assert np.max(np.abs(Ub[d][full] - U1[d][full])) < 1e-9 * scale
