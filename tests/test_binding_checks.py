"""The binding refuses, before any launch, arguments that the PSD-violation
kernels would read or write out of bounds (host-side checks; no GPU needed:
every refusal below happens before the device check)."""
import pytest

torch = pytest.importorskip("torch")


def _args(W_dtype=torch.float64, off_dtype=torch.int32, size_dtype=torch.int32, p=3, n_off=None):
    W = torch.zeros(6 * p, dtype=W_dtype)
    off = torch.zeros(p + 1 if n_off is None else n_off, dtype=off_dtype)
    sizes = torch.full((p,), 3, dtype=size_dtype)
    return W, off, sizes


@pytest.mark.parametrize("fn", ["psd_violation", "psd_violation_noalloc"])
@pytest.mark.parametrize("case", ["W_half", "W_int", "off_int64", "size_int64", "off_short", "empty",
                                  "alpha_f32", "alpha_empty", "noncontig", "cpu"])
def test_violation_refusals(lib, fn, case):
    kw = {}
    if case == "W_half":
        W, off, sizes = _args(W_dtype=torch.float16)
    elif case == "W_int":
        W, off, sizes = _args(W_dtype=torch.int32)
    elif case == "off_int64":
        W, off, sizes = _args(off_dtype=torch.int64)
    elif case == "size_int64":
        W, off, sizes = _args(size_dtype=torch.int64)
    elif case == "off_short":
        W, off, sizes = _args(n_off=3)
    elif case == "empty":
        W, off, sizes = _args(p=0)
    elif case == "noncontig":
        W, off, sizes = _args()
        W = torch.zeros(36, dtype=torch.float64)[::2]
    else:
        W, off, sizes = _args()
    alpha = torch.zeros(1, dtype=torch.float64)
    if case == "alpha_f32":
        alpha = torch.zeros(1, dtype=torch.float32)
    elif case == "alpha_empty":
        alpha = torch.zeros(0, dtype=torch.float64)
    if fn == "psd_violation":
        if case.startswith("alpha"):
            pytest.skip("psd_violation allocates its own alpha")
        call = lambda: lib.psd_violation(W, off, sizes)
    else:
        call = lambda: lib.psd_violation_noalloc(W, off, sizes, alpha)
    with pytest.raises(ValueError):
        call()
