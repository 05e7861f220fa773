"""fw_energy_noalloc (allocation-free energy, static device scratch) against the
handle's own objective evaluation, through the C ABI.  Collected last on
purpose (file name): it must pass after the other GPU tests and alone in a
fresh process."""
import math

import numpy as np
import pytest

from paper_2508_09738_gb300 import binding as B
from paper_2508_09738_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_09738_gb300 import build
    build.build()


def _device_inputs(torch, g, U):
    dev = torch.device("cuda:0")
    return dict(
        rp=torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int32)).to(dev),
        col=torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(dev),
        w=torch.from_numpy(np.ascontiguousarray(g.w, dtype=np.float64)).to(dev),
        U=torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).to(dev),
        lab=torch.from_numpy(np.ascontiguousarray(g.labels, dtype=np.int32)).to(dev),
    )


def _energy(g, d, eps, omega0, laplacian):
    return B.fw_energy_noalloc(g.n, g.K, d["rp"].data_ptr(), d["col"].data_ptr(),
                               d["w"].data_ptr(), g.nnz, d["U"].data_ptr(), g.K,
                               d["lab"].data_ptr(), eps, omega0, laplacian)


@pytest.mark.parametrize("weights,laplacian,tol", [("f64", "sym", 1e-9), ("f32", "sym", 1e-5),
                                                   ("f64", "comb", 1e-9)])
def test_noalloc_energy_matches_handle_objective(weights, laplacian, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = W.blobs_knn(n=1537, K=7, seed=11, label_frac=0.05)   # ragged: 6 tiles of 256 + 1
    eps, omega0 = 50.0, 1000.0
    o = B.fw_seg_default_opts(weight_dtype=weights, laplacian=laplacian, eps=eps, omega0=omega0)
    h = B.fw_seg_create(g.n, g.row_ptr, g.col, g.w, g.K, g.labels, o)
    try:
        B.fw_seg_step(h, 9)                      # a fractional iterate, not U_0
        U = B.fw_seg_get_U(h)
        E_ref = B.fw_seg_objective(h)
    finally:
        B.fw_seg_destroy(h)
    d = _device_inputs(torch, g, U)
    E1 = _energy(g, d, eps, omega0, laplacian)
    E2 = _energy(g, d, eps, omega0, laplacian)   # two calls in a row
    assert math.isfinite(E1)
    assert abs(E1 - E_ref) <= tol * abs(E_ref), (E1, E_ref)
    assert abs(E2 - E_ref) <= tol * abs(E_ref), (E2, E_ref)
    assert E1 == E2                              # exact cross-block sums: reproducible


def test_noalloc_rejects_size_above_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = W.blobs_knn(n=300, K=3, seed=3)
    U = np.full((g.n, g.K), 1.0 / g.K)
    d = _device_inputs(torch, g, U)
    with pytest.raises(B.FwError) as ei:
        # the size check comes before any launch: the small buffers are never read
        B.fw_energy_noalloc(B.FW_NOALLOC_MAX_N + 1, g.K, d["rp"].data_ptr(),
                            d["col"].data_ptr(), d["w"].data_ptr(), g.nnz, d["U"].data_ptr(),
                            g.K, d["lab"].data_ptr(), 50.0, 1000.0)
    assert ei.value.status == B.FW_ERR_UNSUPPORTED
    assert "FW_NOALLOC_MAX_N" in str(ei.value)
    # and a valid call still works afterwards
    assert math.isfinite(_energy(g, d, 50.0, 1000.0, "sym"))
