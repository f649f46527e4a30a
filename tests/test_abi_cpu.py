"""Host-side checks of the C ABI: the library builds, loads, exports every
function declared in include/gmf.h, and rejects bad arguments before any
device work. No compute calls (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as g
    return g


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmf_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(gmf):
    names = declared_functions()
    assert len(names) >= 15
    L = C.CDLL(gmf.LIB_PATH)
    for name in names:
        assert hasattr(L, name), f"{name} declared in gmf.h but not exported"
    assert sorted(gmf.EXPORTS) == names


def test_library_is_sm103a(gmf):
    assert b"sm_103a" in gmf.lib().gmf_version()


def test_config_defaults_are_the_papers(gmf):
    cfg = gmf.gmf_config()
    gmf.lib().gmf_config_default(C.byref(cfg), 100, 50, 2, 1, 5, gmf.GMF_NEGBIN, 10, 10)
    assert (cfg.n, cfg.m, cfg.p, cfg.q, cfg.d, cfg.family) == (100, 50, 2, 1, 5, 1)
    assert list(cfg.lambda_) == [0.0, 0.0, 1.0, 0.0]   # lambda = c(0,0,1,0)
    assert (cfg.k0, cfg.damping, cfg.eps) == (0.01, 1e-3, 1e-8)
    assert (cfg.a1, cfg.a2) == (0.1, 0.01)


def _init(gmf, cfg, **over):
    n, m, p, q, d = cfg.n, cfg.m, cfg.p, cfg.q, cfg.d
    args = dict(Y=np.zeros((n, m), np.int32), X=np.ones((n, p)), Z=np.ones((m, q)),
                rp=np.arange(n, dtype=np.int32), cp=np.arange(m, dtype=np.int32),
                B=np.zeros((m, p)), G=np.zeros((n, q)), U=np.zeros((n, d)), V=np.zeros((m, d)), alpha=1.0)
    args.update(over)
    h = C.c_void_p()
    p_ = lambda a: None if a is None else a.ctypes.data
    rc = gmf.lib().gmf_init(C.byref(h), C.byref(cfg), p_(args["Y"]), 0, 0, None, p_(args["X"]), p_(args["Z"]), None,
                            p_(args["rp"]), p_(args["cp"]), p_(args["B"]), p_(args["G"]), p_(args["U"]),
                            p_(args["V"]), args["alpha"], None)
    return rc, gmf.lib().gmf_last_error().decode()


@pytest.mark.parametrize("field,value,msg", [
    ("n", 0, "positive"), ("d", 70, "1+p+q+d"), ("family", 7, "family"), ("nb_row", 0, "minibatch"),
    ("bias_corr", 2, "bias_corr"), ("alpha_mode", 3, "alpha_mode"), ("precision", 9, "precision"),
    ("a1", 0.0, "a1"), ("k0", -1.0, "learning-rate"), ("flags", 16, "flags"),
])
def test_init_rejects_bad_config(gmf, field, value, msg):
    cfg = gmf.gmf_config()
    gmf.lib().gmf_config_default(C.byref(cfg), 8, 6, 2, 1, 2, 0, 4, 3)
    setattr(cfg, field, value)
    rc, err = _init(gmf, cfg)
    assert rc == gmf.GMF_ERR_ARG
    assert msg in err


@pytest.mark.parametrize("family,y_dtype,alpha_mode,msg", [
    (0, 2, 0, "int32 or uint16 counts"), (1, 2, 0, "int32 or uint16 counts"),
    (2, 0, 0, "float32 responses"), (4, 1, 0, "float32 responses"), (5, 0, 1, "float32 responses"),
    (2, 2, 2, "alpha_mode 2"), (3, 0, 2, "alpha_mode 2"), (6, 2, 0, "unknown family"),
])
def test_init_matches_families_and_response_types(gmf, family, y_dtype, alpha_mode, msg):
    """Counts for the Poisson and NB families, float32 for the Gaussian, Gamma and
    inverse Gaussian (Table S1's supports); per-gene shapes only for the NB."""
    cfg = gmf.gmf_config()
    gmf.lib().gmf_config_default(C.byref(cfg), 8, 6, 2, 1, 2, family, 4, 3)
    cfg.alpha_mode = alpha_mode
    h = C.c_void_p()
    n, m = 8, 6
    Y = np.ones((n, m), np.float32 if y_dtype == 2 else (np.uint16 if y_dtype == 1 else np.int32))
    z = lambda *s: np.zeros(s)
    rc = gmf.lib().gmf_init(C.byref(h), C.byref(cfg), Y.ctypes.data, y_dtype, 0, None, np.ones((n, 2)).ctypes.data,
                            np.ones((m, 1)).ctypes.data, None, np.arange(n, dtype=np.int32).ctypes.data,
                            np.arange(m, dtype=np.int32).ctypes.data, z(m, 2).ctypes.data, z(n, 1).ctypes.data,
                            z(n, 2).ctypes.data, z(m, 2).ctypes.data, 1.0, None)
    assert rc == gmf.GMF_ERR_ARG
    assert msg in gmf.lib().gmf_last_error().decode()


def test_init_rejects_bad_permutation(gmf):
    cfg = gmf.gmf_config()
    gmf.lib().gmf_config_default(C.byref(cfg), 8, 6, 2, 1, 2, 0, 4, 3)
    rc, err = _init(gmf, cfg, rp=np.array([0, 1, 2, 3, 4, 5, 6, 6], np.int32))
    assert rc == gmf.GMF_ERR_ARG and "row_perm" in err
    rc, err = _init(gmf, cfg, cp=np.array([0, 1, 2, 3, 4, 9], np.int32))
    assert rc == gmf.GMF_ERR_ARG and "col_perm" in err
    rc, err = _init(gmf, cfg, alpha=-1.0)
    assert rc == gmf.GMF_ERR_ARG


def test_null_handle_calls_fail_cleanly(gmf):
    L = gmf.lib()
    assert L.gmf_sgd_epoch(None, None, None) == gmf.GMF_ERR_ARG
    assert L.gmf_deviance(None, None, None) == gmf.GMF_ERR_ARG
    assert L.gmf_orthogonalize(None, 1, None) == gmf.GMF_ERR_ARG
    assert L.gmf_num_sweeps(None) == -1
    assert L.gmf_set_wait_limit(None, 0, 0) == gmf.GMF_ERR_ARG
    assert L.gmf_set_flow_lag(None, 2) == gmf.GMF_ERR_ARG
    assert L.gmf_gene_shape_ml(None, None, 10, 1e-6, 1e-3, 1e4, None, None, None) == gmf.GMF_ERR_ARG
    assert L.gmf_fit_loadings(None, 4, None, None) == gmf.GMF_ERR_ARG
    L.gmf_free(None)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle, and fails loudly without libgmf.so."""
    pkg = os.path.join(ROOT, "paper_2412_20509_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src
    src = open(os.path.join(pkg, "__init__.py")).read()
    assert "raise ImportError" in src
