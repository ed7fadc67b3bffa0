"""The C-ABI library builds, loads and exports every entry point that
include/inkjet.h declares; host-side validation rejects bad parameters
before any device work (no GPU needed)."""
import ctypes as C

import pytest

from paper_1702_04487_gb300 import inkjet, workloads as W


def test_library_exports_every_declared_symbol():
    names = inkjet.declared_symbols()
    assert "ij_create" in names and "ij_step" in names and "ij_observe" in names
    lib = C.CDLL(inkjet.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _raw_create(p, count=1):
    arr = (inkjet.ij_params * count)(*([inkjet.make_params(p)] * count))
    out = C.c_void_p(123)
    st = inkjet._lib.ij_create(arr, count, inkjet.ALLOC_FN(), inkjet.FREE_FN(), None, None,
                               C.byref(out))
    return st, out.value


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=-3), dict(rho_ink=1.0, rho_air=1.0), dict(sigma=0.0),
    dict(width_W=-1.0), dict(tau_phi=0.0), dict(nu_air=0.0), dict(theta_deg=181.0),
    dict(geometry=7), dict(axial_bc=5), dict(init_kind=9), dict(precision=3),
    dict(nozzle_width=60, wall_thickness=4), dict(T1=-1), dict(diag_every=-1),
    dict(precision=1, nx=63),  # 2-D FP16 storage pairs columns: nx must be even
])
def test_invalid_parameters_are_rejected_on_the_host(bad):
    p = dict(W.cfg1(), **bad)
    st, out = _raw_create(p)
    assert st == inkjet.IJ_ERR_PARAM
    assert out is None
    assert inkjet.ij_last_error()


def test_null_arguments_and_counts():
    assert inkjet._lib.ij_destroy(None) == inkjet.IJ_OK
    assert inkjet._lib.ij_step(None, 1) == inkjet.IJ_ERR_PARAM
    assert inkjet._lib.ij_time(None, None) == inkjet.IJ_ERR_PARAM
    p = W.cfg1()
    arr = (inkjet.ij_params * 1)(inkjet.make_params(p))
    out = C.c_void_p()
    assert inkjet._lib.ij_create(arr, 0, inkjet.ALLOC_FN(), inkjet.FREE_FN(), None, None,
                                 C.byref(out)) == inkjet.IJ_ERR_PARAM
    assert inkjet._lib.ij_create(arr, 1, inkjet.ALLOC_FN(), inkjet.FREE_FN(), None, None,
                                 None) == inkjet.IJ_ERR_PARAM
    two = [dict(p), dict(p, diag_every=5)]
    arr2 = (inkjet.ij_params * 2)(*[inkjet.make_params(q) for q in two])
    assert inkjet._lib.ij_create(arr2, 2, inkjet.ALLOC_FN(), inkjet.FREE_FN(), None, None,
                                 C.byref(out)) == inkjet.IJ_ERR_PARAM


def test_binding_and_oracle_share_only_the_parameter_names():
    """Both sides take the same parameter dicts (workloads.py) but their
    field lists are written separately; they must agree name for name."""
    from oracle.oracle import _Params
    lib_fields = [f[0] for f in inkjet.ij_params._fields_]
    orc_fields = [f[0] for f in _Params._fields_]
    assert set(orc_fields) <= set(lib_fields)
    assert set(lib_fields) - set(orc_fields) == {"precision", "dim"}


def test_library_exports_every_surrogate_symbol():
    import os
    import re
    with open(os.path.join(os.path.dirname(inkjet.HEADER), "surrogate.h")) as fh:
        names = sorted(set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", fh.read())))
    assert "sg_create" in names and "sg_train" in names and "sg_gemm_bf16" in names
    lib = C.CDLL(inkjet.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_surrogate_config_is_checked_on_the_host():
    from paper_1702_04487_gb300 import surrogate as S
    for bad in (dict(members=0), dict(members=9), dict(hidden=20), dict(hidden=512),
                dict(batch=8), dict(lr=0.0), dict(beta1=1.0), dict(lr_cosine=2)):
        c = dict(S.DEFAULT_CONFIG, **bad)
        conf = S.sg_config(c["members"], c["hidden"], c["batch"], c["lr"], c["beta1"], c["beta2"],
                           c["eps"], c["seed"], c["log_inputs"], c["log_outputs"],
                           (C.c_float * 4)(*c["out_weight"]), c["lr_cosine"])
        out = C.c_void_p(7)
        st = S._lib.sg_create(C.byref(conf), inkjet.ALLOC_FN(), inkjet.FREE_FN(), None, None,
                              C.byref(out))
        assert st == inkjet.IJ_ERR_PARAM and out.value is None
