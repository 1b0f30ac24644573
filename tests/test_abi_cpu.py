"""Host-side checks of the C ABI library (no GPU needed, no compute calls)."""
import ctypes

from paper_1401_4832_gb300 import _build_lib, _native


def test_library_builds_and_exports_every_declared_symbol():
    path = _build_lib.build()
    lib = ctypes.CDLL(path)
    names = _native.header_functions()
    assert set(names) >= {"msa_reweight", "plm_site_objective_grad", "plm_solve",
                          "fn_apc_scores", "plm_create", "plm_destroy",
                          "plm_last_error", "plm_default_opts"}
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/plmdca.h but not exported"


def test_default_opts_follow_the_paper():
    lib = _native.load()
    o = _native.plm_opts()
    lib.plm_default_opts(ctypes.byref(o))
    # recommended inputs of the rundown (Sec. 3.5): x = 0.8, lambda_h = lambda_J = 0.01
    assert (o.x, o.lambda_h, o.lambda_J) == (0.8, 0.01, 0.01)
    assert o.lbfgs_m == 5 and o.gtol == 1e-4 and o.prec == _native.PLM_SPLIT_BF16


def test_struct_sizes_match_header_layout():
    # plm_opts: 4 doubles + 5 ints + 7 reserved ints (+ padding to 8)
    assert ctypes.sizeof(_native.plm_opts) == 4 * 8 + 12 * 4
    assert ctypes.sizeof(_native.plm_report) == 8 * 4 + 5 * 4 + 4
