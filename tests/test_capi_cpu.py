"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol
include/fcgle.h declares, and rejects invalid arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _declared():
    src = open(os.path.join(ROOT, "include", "fcgle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcgle_[a-z_]+)\s*\(", src)))


def test_header_declares_binding_exports(binding):
    assert _declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(binding):
    lib = ctypes.CDLL(binding.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(binding):
    assert binding.fcgle_status_string(0) == "FCGLE_OK"
    assert binding.fcgle_status_string(5) == "FCGLE_ERR_TIMEOUT"


@pytest.mark.parametrize("bad", [
    dict(ns=[0, 4]), dict(alphas=[2.0, 1.5]), dict(alphas=[1.0, 1.5]), dict(nu=0.0), dict(kappa=-1.0),
    dict(boxes=[(1.0, -1.0), (0.0, 1.0)]), dict(fd_order=3), dict(precision=7), dict(ns=[3, 3, 3, 3]),
])
def test_setup_rejects_invalid_parameters(binding, bad):
    args = dict(ns=[4, 5], boxes=[(-1.0, 1.0), (-1.0, 1.0)], alphas=[1.5, 1.5], nu=1.0, eta=0.0,
                gamma=0.0, kappa=1.0, zeta=0.0, fd_order=2, precision="fp64")
    args.update(bad)
    if len(args["ns"]) == 4:
        p = binding.fcgle_params()
        p.d = 4
        h = ctypes.c_void_p()
        st = binding._lib.fcgle_setup(ctypes.byref(p), None, ctypes.byref(h))
        assert st == binding.FCGLE_ERR_INVALID_ARG
        return
    with pytest.raises(binding.FcgleError) as e:
        binding.fcgle_setup(args["ns"], args["boxes"], args["alphas"], args["nu"], args["eta"], args["gamma"],
                            args["kappa"], args["zeta"], args["fd_order"], args["precision"],
                            stream=_FakeStream())
    assert e.value.status == binding.FCGLE_ERR_INVALID_ARG
    assert binding.fcgle_last_error() != ""


def test_null_handle_rejected(binding):
    assert binding._lib.fcgle_step(None, 0, 0.1, 0.0, None) == binding.FCGLE_ERR_INVALID_ARG
    assert binding._lib.fcgle_selftest_bounded_wait(None, None) == binding.FCGLE_ERR_INVALID_ARG
    assert binding._lib.fcgle_destroy(None) == binding.FCGLE_OK


class _FakeStream:
    cuda_stream = 0


def test_tf32_precision_is_reported_unsupported(binding):
    with pytest.raises(binding.FcgleError) as e:
        binding.fcgle_setup([4, 5], [(-1.0, 1.0)] * 2, [1.5, 1.5], 1.0, 0.0, 0.0, 1.0, 0.0,
                            precision=binding.FCGLE_TF32, stream=_FakeStream())
    assert e.value.status == binding.FCGLE_ERR_UNSUPPORTED


@pytest.mark.parametrize("case", ["dtype", "numel", "contiguous", "device"])
def test_norm_static_wrapper_rejects_mismatched_tensors(binding, case):
    """The Python wrapper of fcgle_norm_static checks the tensor against the
    params before the C call (which trusts them); each mismatch is rejected."""
    torch = pytest.importorskip("torch")
    p = binding.make_params([6, 4], [(-1.0, 1.0)] * 2, [1.5, 1.5], 1.0, 0.0, 0.0, 1.0, 0.0, precision="bf16x3")
    u = {"dtype": torch.zeros((4, 6), dtype=torch.complex128),
         "numel": torch.zeros((4, 5), dtype=torch.complex64),
         "contiguous": torch.zeros((6, 4), dtype=torch.complex64).t(),
         "device": torch.zeros((4, 6), dtype=torch.complex64)}[case]
    with pytest.raises(binding.FcgleError) as e:
        binding.fcgle_norm_static(p, u)
    assert e.value.status == binding.FCGLE_ERR_INVALID_ARG
    assert {"dtype": "dtype", "numel": "entries", "contiguous": "contiguous", "device": "CUDA"}[case] in str(e.value)


def test_new_entry_points_reject_null_handles(binding):
    lib = binding._lib
    assert lib.fcgle_set_exp_form(None, 1) == binding.FCGLE_ERR_INVALID_ARG
    s = (ctypes.c_double * 1)(1.0)
    o = (ctypes.c_double * 2)()
    assert lib.fcgle_spectral_scalars(None, 2, 1, 1e-3, 1, s, o, 0) == binding.FCGLE_ERR_INVALID_ARG
    assert lib.fcgle_mode_product(None, 0, 1, None, None) == binding.FCGLE_ERR_INVALID_ARG


def test_autotune_report_without_tuning(binding):
    # nothing has been tuned in this process (no GPU here): the report is empty
    need = ctypes.c_size_t()
    assert binding._lib.fcgle_autotune_report(None, 0, ctypes.byref(need)) == binding.FCGLE_OK
    assert need.value >= 1
    assert isinstance(binding.fcgle_autotune_report(), str)
