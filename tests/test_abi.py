"""The C-ABI library builds, loads and exports every symbol the header
declares; host-only entry points behave without a GPU.  CPU only."""
import ctypes
import os
import re

import pytest

from paper_2202_12808_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "cofem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cofem_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    from paper_2202_12808_gb300 import build
    build.build()
    return B.lib()


def test_header_declares_binding_names():
    assert _header_functions() == B.EXPORTED


def test_library_exports_every_declared_symbol(built):
    for name in _header_functions():
        assert hasattr(built, name), name


def test_status_strings(built):
    assert B.cofem_status_string(0) == "ok"
    assert "workspace" in B.cofem_status_string(7)


def test_params_default_matches_header(built):
    p = B.cofem_params_default()
    assert (p.K, p.em_iters, p.cg_max_iters, p.fixed_cg_iters, p.resid_replace_every) == (20, 50, 400, 0, 0)
    assert p.vec_dtype == B.COFEM_F32
    assert (p.cg_tol, p.alpha_init, p.den_floor, p.support_threshold) == (1e-6, 1.0, 1e-12, 1e6)
    assert p.stop_rule == 0 and p.tasks == 0 and p.solver == 0
    # 8 int32 fields, 4 doubles, seed, t_offset, mlp, solver (padded to 8)
    assert ctypes.sizeof(B.cofem_params) == 8 * 4 + 4 * 8 + 8 + 8 + 8 + 8


def test_stop_rule_validation(built):
    h = B.cofem_op_dense(4, 10, B.COFEM_F32, 256, 64)
    try:
        assert B.cofem_workspace_bytes(h, B.cofem_params_default(stop_rule=1)) > 0
        for bad, code in ((dict(stop_rule=2), 1), (dict(stop_rule=-1), 1),
                          (dict(stop_rule=1, mlp=256), 6)):
            with pytest.raises(B.CofemError) as e:
                B.cofem_workspace_bytes(h, B.cofem_params_default(**bad))
            assert e.value.code == code, bad
    finally:
        B.cofem_op_destroy(h)


def test_solver_validation(built):
    """Block CG (solver 1) takes the joint stop test on its own recurrence:
    residual replacement, the per-column rule and the learned start are
    refused (COFEM_ERR_UNSUPPORTED = 6); other solver values are invalid."""
    h = B.cofem_op_dense(4, 10, B.COFEM_F32, 256, 64)
    try:
        assert B.cofem_workspace_bytes(h, B.cofem_params_default(solver=1)) > \
            B.cofem_workspace_bytes(h, B.cofem_params_default(solver=0))
        for bad, code in ((dict(solver=2), 1), (dict(solver=-1), 1),
                          (dict(solver=1, resid_replace_every=50), 6),
                          (dict(solver=1, stop_rule=1), 6),
                          (dict(solver=1, mlp=256), 6)):
            with pytest.raises(B.CofemError) as e:
                B.cofem_workspace_bytes(h, B.cofem_params_default(**bad))
            assert e.value.code == code, bad
    finally:
        B.cofem_op_destroy(h)


def test_tasks_validation(built):
    h = B.cofem_op_dense(4, 10, B.COFEM_F32, 256, 64)
    try:
        one = B.cofem_workspace_bytes(h, B.cofem_params_default(K=8))
        three = B.cofem_workspace_bytes(h, B.cofem_params_default(K=8, tasks=3))
        assert three > one                       # two more columns per vector block
        for bad, code in ((dict(K=62, tasks=3), 1), (dict(tasks=-1), 1),
                          (dict(tasks=2, mlp=256), 6)):
            with pytest.raises(B.CofemError) as e:
                B.cofem_workspace_bytes(h, B.cofem_params_default(**bad))
            assert e.value.code == code, bad
    finally:
        B.cofem_op_destroy(h)


def test_invalid_operator_arguments(built):
    with pytest.raises(B.CofemError) as e:
        B.cofem_op_dense(0, 10, B.COFEM_F32, 256, 10)
    assert e.value.code == 1
    with pytest.raises(B.CofemError):
        B.cofem_op_dense(4, 10, B.COFEM_F32, 0, 10)          # null pointer
    with pytest.raises(B.CofemError):
        B.cofem_op_dense(4, 10, B.COFEM_BF16, 256, 10)       # ld not a multiple of 64
    with pytest.raises(B.CofemError):
        B.cofem_op_conv1d(100, 8, 64, 256)                   # L not a multiple of 64
    h = B.cofem_op_dense(4, 10, B.COFEM_F32, 256, 12)
    assert B.cofem_op_shape(h) == (4, 10)
    B.cofem_op_destroy(h)
    h = B.cofem_op_conv1d(128, 3, 5, 256)
    assert B.cofem_op_shape(h) == (128, 384)
    B.cofem_op_destroy(h)


def test_conv_tensor_core_switch_and_col_norm_workspace(built):
    # host-side handle logic only (no device memory is touched): the
    # tensor-core switch is accepted for a convolutional handle only, with
    # on in {0, 1}; the column-norm workspace is 0 bytes for a
    # convolutional dictionary and holds the masked DCT's one-column
    # transform scratch plus two D-float buffers
    h = B.cofem_op_conv1d(128, 3, 5, 256)
    try:
        B.cofem_op_conv1d_set_tensor_cores(h, 1)
        B.cofem_op_conv1d_set_tensor_cores(h, 0)
        with pytest.raises(B.CofemError) as e:
            B.cofem_op_conv1d_set_tensor_cores(h, 2)
        assert e.value.code == 1
        assert B.cofem_col_norms_workspace_bytes(h) == 0
    finally:
        B.cofem_op_destroy(h)
    d = B.cofem_op_dct(4096, 1024, 256)
    try:
        with pytest.raises(B.CofemError):
            B.cofem_op_conv1d_set_tensor_cores(d, 1)
        n = B.cofem_col_norms_workspace_bytes(d)
        assert n >= B.cofem_apply_workspace_bytes(d, B.COFEM_F32, 1) + 2 * 4096 * 4
        with pytest.raises(B.CofemError) as e:
            B.cofem_op_col_norms_ws(d, 256, 512, n - 256)   # workspace too small
        assert B.STATUS[e.value.code] == "COFEM_ERR_WORKSPACE"
    finally:
        B.cofem_op_destroy(d)
