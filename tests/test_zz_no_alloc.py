"""mx_dots_noalloc, the allocation-free variant of mx_dots for callers that cannot call
cudaMalloc: a host framework that owns all device memory through its own pool and forbids
side allocations, or an embedding with no allocator to hand the library.

It keeps its block partial sums in a fixed 4 MiB array of the library's device image, so
consecutive calls reuse the same scratch; every call must match mx_dots, which allocates
its scratch per call, to rounding. Above nvec * nrhs of about 860 the array holds fewer
partial-sum blocks than mx_dots uses, so the summation order differs there; the sizes
below cover both sides of that point and the largest allowed size. The file name makes
pytest collect it last."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

mx = pytest.importorskip("paper_1711_03789_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _check(call, nvec, n, nrhs):
    V = torch.from_numpy(inputs.random_complex(100 + call, (nvec, n, nrhs))).cuda()
    w = torch.from_numpy(inputs.random_complex(200 + call, (n, nrhs))).cuda()
    ref = mx.mx_dots(V, w)
    got = mx.mx_dots_noalloc(V, w)
    # rounding bound of an n-term FP64 sum in any order
    bound = 1e-13 * np.sqrt(n) * V.abs().max().item() * w.abs().max().item()
    assert np.abs(got - ref).max() <= bound, (call, nvec, nrhs)
    # device output as well
    hd = torch.zeros((nvec, nrhs), dtype=torch.complex128, device="cuda")
    mx.mx_dots_noalloc(V, w, hd)
    assert np.abs(hd.cpu().numpy() - ref).max() <= bound, (call, nvec, nrhs)


def test_noalloc_matches_allocating_entry_point_twice():
    # two calls in a row with different sizes and data: the second reuses the scratch
    for call, (nvec, n, nrhs) in enumerate([(9, 70001, 16), (3, 5003, 5)]):
        _check(call, nvec, n, nrhs)


def test_noalloc_reduced_block_count_and_largest_size_twice():
    # 27 * 32 = 864 outputs: just above the point where the scratch holds fewer than
    # 2 x SM-count blocks; 512 * 32 = 16384: the largest size, partials nearly fill the
    # array. Each size twice in a row, so the second call reuses what the first left.
    for call, (nvec, n, nrhs) in enumerate([(27, 20011, 32), (27, 20011, 32), (512, 3001, 32), (512, 3001, 32)]):
        _check(10 + call, nvec, n, nrhs)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    V = torch.zeros((1025, 1, 16), dtype=torch.complex128, device="cuda")  # 1025 * 16 > 16384
    w = torch.zeros((1, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(mx.MxError) as e:
        mx.mx_dots_noalloc(V, w)
    assert e.value.code == mx.MX_EINVAL and "16384" in str(e.value)
