"""Input validation of hf_system_create, on CPU: every malformed geometry,
basis or threshold is rejected with its status before the context is used
(the context handle passed here is a zeroed host block, never dereferenced
on these paths)."""
import ctypes

import numpy as np
import pytest

from paper_1708_00033_gb300 import hf
from paper_1708_00033_gb300 import inputs as I


def _create(geom_Z, geom_xyz, atom, l, nprim, exps, coefs, th=(0.0, 0.0, 0.0), ctx=True):
    lib = hf.load_library()
    Z = np.ascontiguousarray(geom_Z, dtype=np.int32)
    xyz = np.ascontiguousarray(geom_xyz, dtype=np.float64)
    at = np.ascontiguousarray(atom, dtype=np.int32)
    ll = np.ascontiguousarray(l, dtype=np.int32)
    npr = np.ascontiguousarray(nprim, dtype=np.int32)
    ex = np.ascontiguousarray(exps, dtype=np.float64)
    co = np.ascontiguousarray(coefs, dtype=np.float64)
    g = hf.Geometry_c(int(Z.shape[0]), Z.ctypes.data_as(hf._i32p), xyz.ctypes.data_as(hf._f64p))
    b = hf.Basis_c(int(ll.shape[0]), at.ctypes.data_as(hf._i32p), ll.ctypes.data_as(hf._i32p),
                   npr.ctypes.data_as(hf._i32p), ex.ctypes.data_as(hf._f64p), co.ctypes.data_as(hf._f64p))
    t = hf.Thresholds_c(*th)
    fake = ctypes.create_string_buffer(4096)
    out = ctypes.c_void_p()
    rc = lib.hf_system_create(ctypes.cast(fake, ctypes.c_void_p) if ctx else None, ctypes.byref(g), ctypes.byref(b),
                              ctypes.byref(t), ctypes.byref(out))
    assert not out.value
    return rc, lib.hf_last_error().decode()


def _water():
    g = I.water_cluster(1, 1, 0)
    b = I.synthetic_basis(g)
    return g, b


def _args(g, b):
    return [g.Z, g.xyz, b.atom, b.l, b.nprim, b.exps, b.coefs]


def test_null_context():
    g, b = _water()
    rc, _ = _create(*_args(g, b), ctx=False)
    assert rc == hf.HF_E_INVALID


@pytest.mark.parametrize("case,code", [
    ("empty_geometry", hf.HF_E_INVALID),
    ("empty_basis", hf.HF_E_INVALID),
    ("negative_charge", hf.HF_E_INVALID),
    ("nan_coordinate", hf.HF_E_INVALID),
    ("atom_out_of_range", hf.HF_E_INVALID),
    ("negative_l", hf.HF_E_INVALID),
    ("sp_without_p_coefficients", hf.HF_E_INVALID),
    ("f_shell", hf.HF_E_UNSUPPORTED),
    ("no_primitives", hf.HF_E_INVALID),
    ("nine_primitives", hf.HF_E_UNSUPPORTED),
    ("zero_exponent", hf.HF_E_INVALID),
    ("nan_coefficient", hf.HF_E_INVALID),
    ("negative_tau", hf.HF_E_INVALID),
    ("negative_prim_tau", hf.HF_E_INVALID),
])
def test_malformed_input_is_rejected(case, code):
    g, b = _water()
    a = [np.array(x, copy=True) for x in _args(g, b)]
    Z, xyz, atom, l, nprim, exps, coefs = a
    th = (1e-10, 0.0, 0.0)
    if case == "empty_geometry":
        Z, xyz = Z[:0], xyz[:0]
    elif case == "empty_basis":
        atom, l, nprim, exps, coefs = atom[:0], l[:0], nprim[:0], exps[:0], coefs[:0]
    elif case == "negative_charge":
        Z[1] = -1
    elif case == "nan_coordinate":
        xyz[2, 1] = np.nan
    elif case == "atom_out_of_range":
        atom[4] = 3
    elif case == "negative_l":
        l[0] = -2
    elif case == "sp_without_p_coefficients":
        l[1] = hf.HF_SP_SHELL  # coefs_p is NULL in _create
    elif case == "f_shell":
        l[5] = 3
    elif case == "no_primitives":
        nprim[2] = 0
    elif case == "nine_primitives":
        nprim = nprim.copy()
        nprim[0] = 9
        exps = np.concatenate([np.full(6, 0.5), exps])
        coefs = np.concatenate([np.full(6, 0.1), coefs])
    elif case == "zero_exponent":
        exps[7] = 0.0
    elif case == "nan_coefficient":
        coefs[3] = np.nan
    elif case == "negative_tau":
        th = (-1e-10, 0.0, 0.0)
    elif case == "negative_prim_tau":
        th = (1e-10, 0.0, -1.0)
    rc, msg = _create(Z, xyz, atom, l, nprim, exps, coefs, th)
    assert rc == code, msg
    assert msg


def test_null_handles_are_rejected():
    """Every entry point answers a NULL handle with HF_E_INVALID (destroy: a no-op), on CPU."""
    lib = hf.load_library()
    n = None
    buf = np.zeros(16)
    p = buf.ctypes.data
    calls = {
        "hf_fock_build": lambda: lib.hf_fock_build(n, p, p, n, n, None, None, 0),
        "hf_fock_build_partial": lambda: lib.hf_fock_build_partial(n, p, 0, 1, p, p, 0),
        "hf_scf_run": lambda: lib.hf_scf_run(n, None, n, n, n, None, None, 0),
        "hf_eigh": lambda: lib.hf_eigh(n, 2, p, p, p, 0),
        "hf_system_set_fock_copies": lambda: lib.hf_system_set_fock_copies(n, 1),
        "hf_measure_peaks": lambda: lib.hf_measure_peaks(n, None),
        "hf_one_electron": lambda: lib.hf_one_electron(n, p, p, 0),
        "hf_system_get_info": lambda: lib.hf_system_get_info(n, None),
        "hf_fock_build_noalloc": lambda: lib.hf_fock_build_noalloc(n, p, p, n, n),
        "hf_fock_build_batch": lambda: lib.hf_fock_build_batch(n, p, p, None, None, 0),
        "hf_batch_tune": lambda: lib.hf_batch_tune(n, None, 0),
        "hf_batch_get_info": lambda: lib.hf_batch_get_info(n, None),
        "hf_batch_offsets": lambda: lib.hf_batch_offsets(n, None),
        "hf_model_create": lambda: lib.hf_model_create(n, n, None),
        "hf_model_get_weights": lambda: lib.hf_model_get_weights(n, n, n),
        "hf_model_forward": lambda: lib.hf_model_forward(n, 1, p, p, 0),
        "hf_model_train_step": lambda: lib.hf_model_train_step(n, 1, p, p, p, 1e-3, None, 0),
        "hf_guess_features": lambda: lib.hf_guess_features(n, n, n, None, 0),
        "hf_guess_predict": lambda: lib.hf_guess_predict(n, n, n, 0),
        "hf_guess_targets": lambda: lib.hf_guess_targets(n, p, p, p, 0),
        "hf_guess_train": lambda: lib.hf_guess_train(n, 1, p, p, p, None, None, 1),
        "hf_fock_assemble": lambda: lib.hf_fock_assemble(n, p, p, p, p, None, 0),
    }
    for name, call in calls.items():
        assert call() == hf.HF_E_INVALID, name
    for name in ("hf_destroy", "hf_system_destroy", "hf_batch_destroy", "hf_model_destroy"):
        getattr(lib, name)(None)
