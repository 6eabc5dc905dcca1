"""The C ABI library builds, loads without a GPU and exports every function declared in include/cdwac.h."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cdwac.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdwac_[A-Za-z_0-9]+)\s*\(", text)))


def test_library_exports_header():
    from paper_2305_15955_gb300 import build, cdwac
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(cdwac.EXPORTED) <= set(names)


def test_default_params_and_errors_without_gpu():
    from paper_2305_15955_gb300 import build, cdwac
    build.build()
    lib = cdwac.load()
    p = cdwac._Params()
    lib.cdwac_default_params(ctypes.byref(p))
    d = cdwac.Params()
    assert (p.n_imag, p.n_real, p.pade_M, p.eta, p.eta_ref) == (d.n_imag, d.n_real, d.pade_M, d.eta, d.eta_ref)
    assert (p.real_set, p.n_core, p.n_val, p.delta_c, p.delta_v) == (d.real_set, d.n_core, d.n_val, d.delta_c,
                                                                      d.delta_v)
    # the library filled the binding's struct up to its last field (zero-initialised before the call)
    assert p.delta_v == 0.5
    # null arguments are rejected on the host, before any CUDA call
    assert lib.cdwac_create(None, 0) == cdwac.ERR_ARG
    assert lib.cdwac_build_W_imag(None, None, None, None, None, None, None) == cdwac.ERR_ARG
    cyc = ctypes.c_int(0)
    assert lib.cdwac_evgw(None, None, None, 0, 0, None, None, 0, 1e-6, 1, None, None, None, ctypes.byref(cyc),
                          None) == cdwac.ERR_ARG
