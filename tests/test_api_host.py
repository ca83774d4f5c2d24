"""Host-side argument handling of the PyTorch wrapper (no GPU): the
precision a transform call selects from its dtype and flags, and the names
of the solver's FP64-accurate arithmetic."""
import pytest

torch = pytest.importorskip("torch")


def test_precision_selection():
    from paper_2306_15511_gb300 import _native as N
    from paper_2306_15511_gb300.api import _prec
    assert _prec(torch.complex128, False) == N.FP64
    assert _prec(torch.float64, False) == N.FP64
    assert _prec(torch.complex64, False) == N.FP32
    assert _prec(torch.complex64, True) == N.TC32
    assert _prec(torch.float32, True) == N.TC32
    assert _prec(torch.complex128, False, True) == N.DF64
    assert _prec(torch.float64, False, True) == N.DF64
    with pytest.raises(ValueError):
        _prec(torch.complex128, True)            # tensor cores need FP32 buffers
    with pytest.raises(ValueError):
        _prec(torch.complex64, False, True)      # double-FP32 needs FP64 buffers
    with pytest.raises(ValueError):
        _prec(torch.complex128, True, True)


def test_fp64_arith_names():
    from paper_2306_15511_gb300 import _native as N
    from paper_2306_15511_gb300.api import _arith
    assert _arith("default") == N.ARITH_DEFAULT
    assert _arith("fp64") == N.ARITH_FP64
    assert _arith("df64") == N.ARITH_DF64
    with pytest.raises(ValueError):
        _arith("quad")
