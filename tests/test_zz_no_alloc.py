"""The PSD-violation entry point that allocates nothing.

Some callers cannot call cudaMalloc when they need the measure: code inside
a framework whose caching allocator owns the device memory, a plugin handed
only its input and output buffers, or a real-time loop that forbids the
latency and possible failure of an allocation.  cdsdp_psd_violation_noalloc
serves them from a fixed device array inside the library.  This test calls it through the C ABI
twice in a row, on two different batches, and checks each result against the
entry point that takes caller scratch, within the tolerance of the other
PSD-violation tests.  The file sorts last so that a run stopping at the first
failure has run every other test before this one."""
import numpy as np
import pytest

from paper_1707_05058_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(rng, count, shift):
    sizes = [int(s) for s in rng.integers(1, 25, count)]
    blocks = []
    for s in sizes:
        G = W._f32(rng.standard_normal((s, s)))
        blocks.append(W._f32(G @ G.T - shift * np.eye(s)))
    packed = np.concatenate([np.concatenate([B[b:, b] for b in range(B.shape[0])]) for B in blocks])
    off = np.concatenate([[0], np.cumsum([s * (s + 1) // 2 for s in sizes])])
    return blocks, sizes, packed, off


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_scratch_entry_point(lib, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 2e-5
    rng = np.random.default_rng(2024 if prec == "fp64" else 2025)
    for call, (count, shift) in enumerate([(1500, 2.0), (37, 0.25)]):
        blocks, sizes, packed, off = _batch(rng, count, shift)
        Wd = torch.tensor(packed, dtype=dt, device="cuda")
        offd = torch.tensor(off, dtype=torch.int32, device="cuda")
        szd = torch.tensor(sizes, dtype=torch.int32, device="cuda")
        alpha = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        lib.psd_violation_noalloc(Wd, offd, szd, alpha)
        ref = lib.psd_violation(Wd, offd, szd)
        torch.cuda.synchronize()
        a, r = alpha.item(), ref.item()
        scale = max(1.0, max(np.linalg.norm(B) for B in blocks))
        assert abs(a - r) <= tol * scale, (call, a, r)
        want = -min(0.0, min(np.linalg.eigvalsh(B).min() for B in blocks))
        assert abs(a - want) <= tol * scale, (call, a, want)


def test_noalloc_rejects_oversize(lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = 524160 + 4
    sizes = torch.ones(p, dtype=torch.int32, device="cuda")
    off = torch.arange(p + 1, dtype=torch.int32, device="cuda")
    Wd = torch.ones(p, dtype=torch.float64, device="cuda")
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.CdsdpError) as e:
        lib.psd_violation_noalloc(Wd, off, sizes, alpha)
    assert e.value.status == -8


@pytest.mark.parametrize("noalloc", [True, False])
def test_order_out_of_range_gives_nan(lib, noalloc):
    """An order outside 1..max_size (here 0) is not a valid block: alpha comes
    out NaN instead of silently ignoring the block."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(7)
    blocks, sizes, packed, off = _batch(rng, 9, 0.5)
    sizes = list(sizes)
    sizes[4] = 0  # its packed entries are still read by nobody: offsets unchanged
    Wd = torch.tensor(packed, dtype=torch.float64, device="cuda")
    offd = torch.tensor(off, dtype=torch.int32, device="cuda")
    szd = torch.tensor(sizes, dtype=torch.int32, device="cuda")
    if noalloc:
        alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
        lib.psd_violation_noalloc(Wd, offd, szd, alpha)
    else:
        alpha = lib.psd_violation(Wd, offd, szd)
    torch.cuda.synchronize()
    assert np.isnan(alpha.item())
