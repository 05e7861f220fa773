"""fw_energy_noalloc, the allocation-free energy evaluation, through the C ABI.

Callers that cannot allocate device memory (a process whose free HBM is held
by another allocator, a loop that must not call cudaMalloc / cudaFree) use it
on a graph and an iterate already in their own device memory; its only
scratch is a fixed-size static device array.  It is checked here against the
FP64 oracle's energy and against a handle's own objective, on two calls in a
row each time.  Collected last on purpose (file name): it must pass after the
other GPU tests and alone in a fresh process."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2508_09738_gb300 import binding as B
from paper_2508_09738_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_09738_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to("cuda:0")


def _device_inputs(torch, g, U, labels=None):
    return dict(rp=_dev(torch, g.row_ptr, np.int32), col=_dev(torch, g.col, np.int32),
                w=_dev(torch, g.w, np.float64), U=_dev(torch, U, np.float64),
                lab=_dev(torch, g.labels if labels is None else labels, np.int32))


def _energy(g, d, eps, omega0, laplacian, ldu=None, labels=True, nnz=None):
    return B.fw_energy_noalloc(g.n, g.K, d["rp"].data_ptr(), d["col"].data_ptr(),
                               d["w"].data_ptr(), g.nnz if nnz is None else nnz,
                               d["U"].data_ptr(), g.K if ldu is None else ldu,
                               d["lab"].data_ptr() if labels else 0, eps, omega0, laplacian)


def _random_U(g, seed):
    return np.random.default_rng(seed).dirichlet(np.ones(g.K), size=g.n)


@pytest.mark.parametrize("weights,laplacian,tol", [("f64", "sym", 1e-9), ("f32", "sym", 1e-5),
                                                   ("f64", "comb", 1e-9)])
def test_noalloc_energy_matches_handle_objective(torch, weights, laplacian, tol):
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


@pytest.mark.parametrize("laplacian", ["sym", "comb"])
def test_noalloc_energy_matches_oracle(torch, laplacian):
    """FP64 against the oracle's E(U) on the same FP64 weights (L_s or D - W):
    the normalised weights are formed by the same IEEE operations, so only the
    summation order differs."""
    g = W.blobs_knn(n=2000, K=5, seed=31, label_frac=0.05)
    U = _random_U(g, 1)
    P = O.make_problem(g, 50.0, 1000.0, "f64", kind=laplacian)
    E_o = O.energy(U, P)
    d = _device_inputs(torch, g, U)
    for _ in range(2):
        E = _energy(g, d, 50.0, 1000.0, laplacian)
        assert abs(E - E_o) <= 1e-12 * abs(E_o), (E, E_o)


def test_noalloc_energy_large_n_grid_stride(torch):
    """n = 300,000 rows: more rows than the 1024 x 256 threads of the capped
    grid, so the grid-stride loops of both kernels take some rows twice."""
    g = W.sbm(n=300_000, K=10, deg_in=20.0, deg_out=2.0, label_frac=0.01, seed=12)
    assert g.n > 1024 * 256
    U = _random_U(g, 2)
    P = O.make_problem(g, 50.0, 1000.0, "f64")
    E_o = O.energy(U, P)
    d = _device_inputs(torch, g, U)
    E1 = _energy(g, d, 50.0, 1000.0, "sym")
    E2 = _energy(g, d, 50.0, 1000.0, "sym")
    assert E1 == E2
    assert abs(E1 - E_o) <= 1e-12 * abs(E_o), (E1, E_o)


def test_noalloc_padded_rows_and_no_labels(torch):
    """A row stride ldu = K + 3 whose padding holds NaN (never read), and
    labels_dev = NULL (no fidelity node), against the oracle's energy with
    every node unlabelled."""
    g = W.blobs_knn(n=777, K=4, seed=41, label_frac=0.05)
    U = _random_U(g, 3)
    Upad = np.full((g.n, g.K + 3), np.nan)
    Upad[:, :g.K] = U
    g0 = W.Graph(g.n, g.row_ptr, g.col, g.w, g.K, np.full(g.n, -1, np.int32), g.truth)
    E_o = O.energy(U, O.make_problem(g0, 50.0, 1000.0, "f64"))
    d = _device_inputs(torch, g, Upad)
    for _ in range(2):
        E = _energy(g, d, 50.0, 1000.0, "sym", ldu=g.K + 3, labels=False)
        assert abs(E - E_o) <= 1e-12 * abs(E_o), (E, E_o)


def test_noalloc_flagged_errors_then_valid_call(torch):
    """Errors found on the device (column out of range, a row extent beyond
    nnz, a node of degree 0, a label >= K) are reported, and each is followed
    by a valid call that must give the oracle's energy: the error word and the
    accumulators of the shared scratch start from zero on every call."""
    g = W.blobs_knn(n=64, K=3, seed=2, label_frac=0.1)
    U = _random_U(g, 4)
    E_o = O.energy(U, O.make_problem(g, 50.0, 1000.0, "f64"))
    good = _device_inputs(torch, g, U)

    def valid():
        for _ in range(2):
            E = _energy(g, good, 50.0, 1000.0, "sym")
            assert abs(E - E_o) <= 1e-12 * abs(E_o), (E, E_o)

    valid()
    cases = []
    col = g.col.copy()
    col[5] = g.n + 5
    cases.append((_device_inputs(torch, W.Graph(g.n, g.row_ptr, col, g.w, g.K, g.labels,
                                                g.truth), U), g.nnz, B.FW_ERR_GRAPH))
    rp = g.row_ptr.copy()
    rp[-1] = g.nnz + 4                    # last row reaches past nnz (never read there)
    cases.append((_device_inputs(torch, W.Graph(g.n, rp, g.col, g.w, g.K, g.labels, g.truth),
                                 U), g.nnz, B.FW_ERR_GRAPH))
    w0 = g.w.copy()
    w0[g.row_ptr[3]:g.row_ptr[4]] = 0.0   # node 3: degree 0
    cases.append((_device_inputs(torch, W.Graph(g.n, g.row_ptr, g.col, w0, g.K, g.labels,
                                                g.truth), U), g.nnz, B.FW_ERR_ISOLATED))
    lab = g.labels.copy()
    lab[9] = g.K
    cases.append((_device_inputs(torch, g, U, labels=lab), g.nnz, B.FW_ERR_INVALID_ARG))
    for d, nnz, want in cases:
        with pytest.raises(B.FwError) as e:
            _energy(g, d, 50.0, 1000.0, "sym", nnz=nnz)
        assert e.value.status == want
        valid()


def test_noalloc_rejects_size_above_limit(torch):
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
