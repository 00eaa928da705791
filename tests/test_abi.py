"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/lqcd.h, sizes are consistent, and invalid arguments are
rejected on the host before any CUDA call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lqcd.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def api():
    from paper_1512_03487_gb300 import api as a
    return a


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for n in ("lqcd_dslash", "lqcd_M", "lqcd_MdagM", "lqcd_cg_solve", "lqcd_force", "lqcd_spinor_pack"):
        assert n in names


def test_library_exports_every_declared_symbol(api):
    names = _declared_functions()
    missing = [n for n in names if not hasattr(api.lib, n)]
    assert not missing, missing
    # and the Python binding wraps each one under the same name
    from paper_1512_03487_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == names


def test_version_and_counter(api):
    assert "sm_103a" in api.lqcd_version()
    assert api.lqcd_launch_count() >= 0


def test_sizes(api):
    lat = api.lattice((4, 4, 4, 4))
    vh = 128
    assert api.lqcd_spinor_bytes(lat, api.LQCD_F64, api.LQCD_EVEN) == vh * 192
    assert api.lqcd_spinor_bytes(lat, api.LQCD_F32, api.LQCD_FULL) == 2 * vh * 96
    assert api.lqcd_spinor_bytes(lat, api.LQCD_F16, api.LQCD_ODD) == vh * 52
    assert api.lqcd_gauge_bytes(lat, api.LQCD_F32, 12) == 8 * vh * 48
    assert api.lqcd_gauge_bytes(lat, api.LQCD_F64, 18) == 8 * vh * 144
    # ragged: Vh = 6 * 2 * 2 * 6 / 2 = 72 sites, padded to 96 per checkerboard
    lat2 = api.lattice((6, 2, 2, 6), n5=1)
    assert api.lqcd_spinor_bytes(lat2, api.LQCD_F32, api.LQCD_EVEN) == 96 * 96
    # invalid geometry -> 0
    assert api.lqcd_spinor_bytes(api.lattice((5, 4, 4, 4)), api.LQCD_F32, api.LQCD_EVEN) == 0
    assert api.lqcd_spinor_bytes(lat, 7, api.LQCD_EVEN) == 0


def test_workspace_queries(api):
    lat = api.lattice((4, 4, 4, 8))
    op = api.operator(mass=0.1)
    prm = api.solver_params(sloppy_prec=api.LQCD_F16, sloppy_recon=12)
    ws_even = api.lqcd_cg_workspace_bytes(lat, op, prm, api.LQCD_EVEN)
    ws_full = api.lqcd_cg_workspace_bytes(lat, op, prm, api.LQCD_FULL)
    assert 0 < ws_even < ws_full
    assert api.lqcd_operator_workspace_bytes(lat, op, api.LQCD_EVEN) > 0
    bad = api.solver_params(tol=-1.0)
    assert api.lqcd_cg_workspace_bytes(lat, op, bad, api.LQCD_EVEN) == 0
    # the intermediate replacement level reuses the FP64 update's buffers: no extra workspace
    mid = api.solver_params(sloppy_prec=api.LQCD_F16, sloppy_recon=12, delta=1e-5, delta_mid=0.003)
    assert api.lqcd_cg_workspace_bytes(lat, op, mid, api.LQCD_EVEN) == ws_even
    for d in (-0.1, 1.0, float("nan")):
        assert api.lqcd_cg_workspace_bytes(lat, op, api.solver_params(delta_mid=d), api.LQCD_EVEN) == 0


def test_fma_probe_is_outside_the_abi_and_rejects_bad_arguments(api):
    """The bench's FMA probe lives in its own library, not in liblqcd, and
    validates its arguments on the host before any launch."""
    import ctypes as C
    from paper_1512_03487_gb300 import measure
    assert not hasattr(api.lib, "lqcd_fma_probe") or _not_exported(api.lib, "lqcd_fma_probe")
    lib = measure.lib()
    assert lib.fma_probe(None, 0, 10, 1, None) == -1
    assert lib.fma_probe(C.c_void_p(4096), 2, 10, 1, None) == -1  # FP16 is not a probe precision
    assert lib.fma_probe(C.c_void_p(4096), 0, 0, 1, None) == -1
    assert lib.fma_probe(C.c_void_p(4100), 0, 10, 1, None) == -1  # misaligned


def _not_exported(lib, name):
    try:
        getattr(lib, name)
        return False
    except AttributeError:
        return True


def test_struct_layouts_match_the_header(api):
    """The ctypes mirrors of the C structs end where the header's do: the
    fields appended last (delta_mid, update_prec, residual_replacements) sit
    at their C offsets, so older callers that zero the struct keep working."""
    import ctypes as C
    from paper_1512_03487_gb300 import _lib
    P = _lib.lqcd_solver_params
    assert P.delta_mid.offset == P.timeout_ms.offset + 8 and P.update_prec.offset == P.delta_mid.offset + 8
    assert P.reserved.offset == P.update_prec.offset + 4 and C.sizeof(P) == P.reserved.offset + 4
    I = _lib.lqcd_solve_info
    assert I.residual_replacements.offset == I.status.offset + 4


@pytest.mark.parametrize("case", ["odd_lx", "odd_lz", "bad_bc", "bad_prec", "bad_recon", "null", "alias", "n5"])
def test_invalid_arguments_rejected_on_host(api, case):
    """Each call below fails in argument validation, before any CUDA call."""
    lat = api.lattice((4, 4, 4, 4))
    op = api.operator(mass=0.1, prec=api.LQCD_F32)
    buf = 4096  # a fake, 16-byte aligned address never dereferenced
    if case == "odd_lx":
        lat = api.lattice((3, 4, 4, 4))
    elif case == "odd_lz":
        lat = api.lattice((4, 4, 5, 4))  # a hop wrapping in z would keep its parity
    elif case == "bad_bc":
        lat = api.lattice((4, 4, 4, 4), bc=(1, 1, 1, 0.5))
    elif case == "bad_prec":
        op = api.operator(prec=5)
    elif case == "bad_recon":
        op = api.operator(recon=8)
    elif case == "n5":
        lat = api.lattice((4, 4, 4, 4), n5=0)
    args = (buf, buf + 4096 if case != "alias" else buf, buf + 8192)
    if case == "null":
        args = (0, buf, buf)
    with pytest.raises(api.LqcdError) as ei:
        api.lqcd_dslash(args[0], args[1], args[2], lat, op, api.LQCD_EVEN, 0, stream=0)
    assert ei.value.status == -1
    assert api.lqcd_last_error()


def test_cg_rejects_bad_arguments_on_host(api):
    lat = api.lattice((4, 4, 4, 4))
    op = api.operator(prec=api.LQCD_F32)  # CG needs LQCD_F64 outer fields
    prm = api.solver_params()
    info = api.lqcd_solve_info()
    st = api.lib.lqcd_cg_solve(4096, 8192, 12288, 12288, C.byref(lat), C.byref(op), C.byref(prm),
                               api.LQCD_EVEN, C.byref(info), 1 << 20, 1 << 30, None)
    assert st == -1 and info.status == -1
    op = api.operator()
    st = api.lib.lqcd_cg_solve(4096, 8192, 12288, 12288, C.byref(lat), C.byref(op), C.byref(prm),
                               api.LQCD_EVEN, C.byref(info), 1 << 20 | 16, 1 << 30, None)
    assert st == -1  # workspace not 256-byte aligned
    st = api.lib.lqcd_cg_solve(4096, 8192, 12288, 12288, C.byref(lat), C.byref(op), C.byref(prm),
                               api.LQCD_EVEN, C.byref(info), 1 << 20, 16, None)
    assert st == -7  # workspace too small


def test_colour_matrix_sizes_and_rejections(api):
    lat = api.lattice((4, 4, 4, 6), n5=3)  # 1152 sites, padded to 1152
    assert api.lqcd_colour_matrix_bytes(lat, api.LQCD_F64) == 1152 * 144
    assert api.lqcd_colour_matrix_bytes(lat, api.LQCD_F32) == 1152 * 72
    assert api.lqcd_colour_matrix_bytes(api.lattice((2, 2, 2, 6), n5=1), api.LQCD_F32) == 64 * 72  # 48 -> 64
    assert api.lqcd_colour_matrix_bytes(lat, api.LQCD_F16) == 0
    buf = 4096
    for z, x, y, prec in ((buf, buf, buf, api.LQCD_F16), (0, buf, buf, api.LQCD_F32),
                          (buf + 8, buf, buf, api.LQCD_F64)):
        with pytest.raises(api.LqcdError) as ei:
            api.lqcd_su3_mul(z, x, y, lat, prec, stream=0)
        assert ei.value.status == -1


def test_gparity_rejected_on_host(api):
    lat1 = api.lattice((4, 4, 4, 4), n5=1)
    lat2 = api.lattice((4, 4, 4, 4), n5=2)
    buf = 4096
    for lat, op in ((lat1, api.operator(gparity=1)),            # n5 must be 2 flavours
                    (lat2, api.operator(prec=2, gparity=1)),    # FP16 storage
                    (lat2, api.operator(kind=1, gparity=1)),    # domain wall
                    (lat2, api.operator(gparity=16))):          # mask beyond t
        with pytest.raises(api.LqcdError) as ei:
            api.lqcd_dslash(buf, buf + 8192, buf + 16384, lat, op, api.LQCD_EVEN, 0, stream=0)
        assert ei.value.status in (-1, -6)


def test_tune_table_file_format_on_host(api, tmp_path):
    """The autotuner's table (text key -> choice) is host state: load keeps
    values in 0..64 with a tab separator (CRLF tolerated, the last value of a
    repeated key wins; 0 is a hop launch-shape index), save writes them back
    one per line and lqcd_tune_get reads one entry (-1 when absent)."""
    n0 = api.lqcd_tune_entries()
    src = tmp_path / "tune_in.txt"
    src.write_bytes(b"4\thost-test-a\n0\thost-test-zero\n65\thost-test-big\n-1\thost-test-neg\n"
                    b"no separator here\nx\thost-test-nan\n8\thost-test-b\r\n\n3\thost-test-a\n")
    api.lqcd_tune_load(str(src))
    assert api.lqcd_tune_entries() == n0 + 3
    assert api.lqcd_tune_get("host-test-a") == 3
    assert api.lqcd_tune_get("host-test-zero") == 0
    assert api.lqcd_tune_get("host-test-big") == -1
    out = tmp_path / "tune_out.txt"
    api.lqcd_tune_save(str(out))
    lines = out.read_text().splitlines()
    assert len(lines) == n0 + 3
    assert "3\thost-test-a" in lines and "8\thost-test-b" in lines and "0\thost-test-zero" in lines
    assert not any(k in ln for ln in lines for k in ("host-test-big", "host-test-neg", "host-test-nan"))
    with pytest.raises(api.LqcdError):
        api.lqcd_tune_load(str(tmp_path / "missing.txt"))
    with pytest.raises(api.LqcdError):
        api.lqcd_tune_save(str(tmp_path))  # a directory cannot be opened for writing


def test_autograd_rejects_host_tensors(api):
    """FermionAction wants complex128 CUDA tensors; CPU or real inputs fail before any library call."""
    import torch
    from paper_1512_03487_gb300 import autograd
    U = torch.zeros((4, 2, 2, 2, 4, 3, 3), dtype=torch.complex128)
    phi = torch.zeros((4, 2, 2, 2, 4, 3), dtype=torch.complex128)
    with pytest.raises(TypeError):
        autograd.fermion_action(U, phi, 0.1)
    with pytest.raises(TypeError):
        autograd.fermion_action(U.real, phi.real, 0.1)


def test_double_float_operator_rejections_on_host(api):
    """LQCD_F64_DF serves Wilson without G-parity and domain wall on 18-real
    links with L_s dividing 32: domain wall with L_s = 6 or 12-real links and
    G-parity are refused before any CUDA call, and a solver's update_prec
    accepts only LQCD_F64 and LQCD_F64_DF."""
    buf = 4096
    for n5, recon in ((6, 18), (4, 12)):
        lat5 = api.lattice((4, 4, 4, 4), n5=n5)
        with pytest.raises(api.LqcdError) as ei:
            api.lqcd_dslash(buf, buf + 8192, buf + 16384, lat5,
                            api.operator(kind=api.LQCD_DWF, prec=api.LQCD_F64_DF, recon=recon), api.LQCD_EVEN, 0,
                            stream=0)
        assert ei.value.status == -6
    lat2 = api.lattice((4, 4, 4, 4), n5=2)
    with pytest.raises(api.LqcdError) as ei:
        api.lqcd_dslash(buf, buf + 8192, buf + 16384, lat2, api.operator(prec=api.LQCD_F64_DF, gparity=1),
                        api.LQCD_EVEN, 0, stream=0)
    assert ei.value.status == -6
    lat = api.lattice((4, 4, 4, 4))
    op = api.operator()
    assert api.lqcd_cg_workspace_bytes(lat, op, api.solver_params(sloppy_prec=1, update_prec=api.LQCD_F64_DF),
                                       api.LQCD_EVEN) > 0
    assert api.lqcd_cg_workspace_bytes(lat, op, api.solver_params(sloppy_prec=1, update_prec=2), api.LQCD_EVEN) == 0
    # the layout of a double-float operator's fields is the FP64 one
    assert api.lqcd_operator_workspace_bytes(lat, api.operator(prec=api.LQCD_F64_DF), api.LQCD_EVEN) == \
        api.lqcd_operator_workspace_bytes(lat, api.operator(prec=api.LQCD_F64), api.LQCD_EVEN)
