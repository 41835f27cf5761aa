"""mx_dots_noalloc, the allocation-free variant of mx_dots for callers that cannot call
cudaMalloc (a framework that owns all device memory, code between CUDA-graph recordings).

It keeps its block partial sums in a fixed 4 MiB array of the library's device image, so
two calls in a row reuse the same scratch; both must match mx_dots, which allocates its
scratch per call. The file name makes pytest collect it last."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

mx = pytest.importorskip("paper_1711_03789_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_noalloc_matches_allocating_entry_point_twice():
    # two calls in a row with different sizes and data: the second reuses the scratch
    for call, (nvec, n, nrhs) in enumerate([(9, 70001, 16), (3, 5003, 5)]):
        V = torch.from_numpy(inputs.random_complex(100 + call, (nvec, n, nrhs))).cuda()
        w = torch.from_numpy(inputs.random_complex(200 + call, (n, nrhs))).cuda()
        ref = mx.mx_dots(V, w)
        got = mx.mx_dots_noalloc(V, w)
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-13 * scale, call
        # device output as well
        hd = torch.zeros((nvec, nrhs), dtype=torch.complex128, device="cuda")
        mx.mx_dots_noalloc(V, w, hd)
        assert np.abs(hd.cpu().numpy() - ref).max() <= 1e-13 * scale


def test_noalloc_rejects_sizes_beyond_the_scratch():
    V = torch.zeros((1025, 1, 16), dtype=torch.complex128, device="cuda")  # 1025 * 16 > 16384
    w = torch.zeros((1, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(mx.MxError) as e:
        mx.mx_dots_noalloc(V, w)
    assert e.value.code == mx.MX_EINVAL and "16384" in str(e.value)
