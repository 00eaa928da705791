"""Batched CG over uneven lattices in one persistent launch per phase: every
instance must reach its own FP64 true residual, recomputed by the oracle."""
import os

import numpy as np
import pytest

from oracle import cg as ocg
from oracle import wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import from_cb, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _setup(L, shapes, masses, sloppy, recon_s):
    F = L.fields
    entries, keep = [], []
    for k, (dims, m) in enumerate(zip(shapes, masses)):
        lat = L.lattice(dims, bc=BC)
        U = gauge_field(dims, "haar", 500 + k)
        b = to_cb(gaussian_spinor(dims, 600 + k, lead=(1,)), 0)
        g64 = F.gauge_to_device(U, lat, 0, 18)
        gs = F.gauge_to_device(U, lat, sloppy, recon_s) if sloppy else None
        x = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
        bd = F.spinor_to_device(b, lat, 0, 0)
        entries.append(dict(lat=lat, mass=m, gauge=g64, gauge_sloppy=gs, x=x, b=bd))
        keep.append((U, b, lat, dims, m))
    return entries, keep


@pytest.mark.parametrize("sloppy,recon_s,update_prec", [(0, 18, 0), (1, 12, 0), (2, 12, 0), (1, 12, 3), (2, 12, 3)])
def test_uneven_batch_reaches_tolerance(L, sloppy, recon_s, update_prec):
    """FP64, FP32 and FP16 inner operators; reliable updates on the FP64 pipe or
    in double-float arithmetic (update_prec 3)."""
    shapes = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 4, 4, 8), (4, 4, 2, 2), (6, 6, 6, 6)]
    masses = [0.05, 0.05, 0.1, 0.2, 0.01]
    entries, keep = _setup(L, shapes, masses, sloppy, recon_s)
    items = L.batch_items(entries)
    prm = L.solver_params(tol=1e-10, maxiter=3000, sloppy_prec=sloppy, sloppy_recon=recon_s, delta=0.01,
                          check_interval=32, update_prec=update_prec)
    ws = L.fields.empty(L.lqcd_batch_cg_workspace_bytes(len(entries), items, 18, prm))
    infos = L.lqcd_batch_cg_solve(len(entries), items, 18, prm, ws)
    for e, (U, b, lat, dims, m), info in zip(entries, keep, infos):
        assert info.status == 0
        x = L.fields.spinor_to_host(e["x"], lat, 0, 0)
        res = ocg.true_residual(lambda v: wilson.schur_dag_schur(U, v, m, BC), from_cb(x, 0), from_cb(b, 0))
        assert res <= 1e-10, (dims, m, res)
        assert info.true_rel_residual <= 1e-10
    # a second solve of the same shape reuses the tuned grid and the cached graph
    infos2 = L.lqcd_batch_cg_solve(len(entries), items, 18, prm, ws)
    assert infos2[0].iterations == infos[0].iterations


def test_batch_matches_single_solves(L):
    shapes = [(4, 4, 4, 4), (8, 4, 4, 4)]
    masses = [0.05, 0.1]
    entries, keep = _setup(L, shapes, masses, 0, 18)
    items = L.batch_items(entries)
    prm = L.solver_params(tol=1e-12, maxiter=3000)
    ws = L.fields.empty(L.lqcd_batch_cg_workspace_bytes(2, items, 18, prm))
    L.lqcd_batch_cg_solve(2, items, 18, prm, ws)
    F = L.fields
    for e, (U, b, lat, dims, m) in zip(entries, keep):
        op = L.operator(mass=m)
        x1 = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
        ws1 = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 0))
        L.lqcd_cg_solve(x1, e["b"], e["gauge"], e["gauge"], lat, op, prm, 0, ws1)
        a = F.spinor_to_host(e["x"], lat, 0, 0)
        c = F.spinor_to_host(x1, lat, 0, 0)
        assert np.linalg.norm(a - c) <= 1e-10 * np.linalg.norm(c)


def test_tune_table_roundtrip(L, tmp_path):
    entries, _ = _setup(L, [(4, 4, 2, 2), (2, 2, 2, 4)], [0.3, 0.3], 0, 18)
    items = L.batch_items(entries)
    prm = L.solver_params(tol=1e-8, maxiter=500)
    L.lqcd_batch_cg_solve(2, items, 18, prm, L.fields.empty(L.lqcd_batch_cg_workspace_bytes(2, items, 18, prm)))
    n0 = L.lqcd_tune_entries()
    assert n0 >= 1  # the solve above tuned its batch shape
    path = str(tmp_path / "tune.txt")
    L.lqcd_tune_save(path)
    lines = open(path).read().strip().splitlines()
    assert len(lines) == n0 and all("\t" in ln for ln in lines)
    L.lqcd_tune_load(path)
    assert L.lqcd_tune_entries() == n0
    assert os.path.getsize(path) > 0


@pytest.mark.parametrize("tile", [0, 1, 2])
def test_forced_tile_sizes(L, tmp_path, tile):
    """A loaded table that sets the batch's tile size (64, 128 or 256 sites per
    block, key "batch_tile ...") and its grid (key "batch_hop ...") changes the
    launch; every instance still reaches the oracle-recomputed FP64 residual,
    and the loaded entries are not re-timed."""
    shapes = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 4, 4, 8)]
    masses = [0.05, 0.05, 0.1]
    entries, keep = _setup(L, shapes, masses, 1, 12)
    items = L.batch_items(entries)
    prm = L.solver_params(tol=1e-10, maxiter=3000, sloppy_prec=1, sloppy_recon=12, delta=0.01, check_interval=32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tail = f"sms={sms} prec=1 recon=12 : " + " ".join("x".join(map(str, d)) for d in shapes)
    path = tmp_path / "batch_tune.txt"
    path.write_text(f"{tile}\tbatch_tile {tail}\n2\tbatch_hop {tail}\n")
    L.lqcd_tune_load(str(path))
    L.lqcd_release_caches()
    ws = L.fields.empty(L.lqcd_batch_cg_workspace_bytes(len(entries), items, 18, prm))
    infos = L.lqcd_batch_cg_solve(len(entries), items, 18, prm, ws)
    assert L.lqcd_tune_get(f"batch_tile {tail}") == tile and L.lqcd_tune_get(f"batch_hop {tail}") == 2
    for e, (U, b, lat, dims, m), info in zip(entries, keep, infos):
        assert info.status == 0
        x = L.fields.spinor_to_host(e["x"], lat, 0, 0)
        res = ocg.true_residual(lambda v: wilson.schur_dag_schur(U, v, m, BC), from_cb(x, 0), from_cb(b, 0))
        assert res <= 1e-10, (tile, dims, m, res)
