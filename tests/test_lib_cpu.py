"""CPU-side checks of the CUDA library and its binding (no GPU needed)."""
import ast
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2508_09738_gb300")


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(fw_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2508_09738_gb300 import build as B
    return B.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (fw_\w+)", out))
    decl = declared_functions()
    assert decl, "no declarations found"
    missing = [d for d in decl if d not in exported]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2508_09738_gb300 import binding as Bd
    Bd.lib()  # loads without a GPU
    for name in declared_functions():
        assert hasattr(Bd.lib(), name)
        assert hasattr(Bd, name) or name in Bd._SIGS, name


def test_defaults_and_footprint(libpath):
    from paper_2508_09738_gb300 import binding as Bd
    o = Bd.fw_seg_default_opts()
    assert (o.eps, o.omega0, o.max_iters, o.weight_dtype, o.oracle, o.step_rule) == \
        (50.0, 1000.0, 500, 0, 0, 0)
    f32 = Bd.fw_seg_footprint(200_000, 4_400_000, 10, "f32")
    bf16 = Bd.fw_seg_footprint(200_000, 4_400_000, 10, "bf16")
    assert bf16 < f32
    # at least CSR + the three iterate arrays
    assert f32 > 4_400_000 * 8 + 3 * 4 * 200_000 * 10
    # the server's shared epochs default to per-item launches; a schedule
    # outside the enum is rejected before any device call
    so = Bd.fw_srv_default_opts()
    assert so.schedule == Bd.SCHED["items"]
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_srv_create(Bd.fw_srv_default_opts(schedule=7))
    assert e.value.status == Bd.FW_ERR_INVALID_ARG


def test_create_without_gpu_reports_cuda_error(libpath):
    """No silent CPU fallback: without a device the call fails with a status."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2508_09738_gb300 import binding as Bd
    from paper_2508_09738_gb300 import workloads as W
    g = W.blobs_knn(n=50, K=3, seed=1)
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(g.n, g.row_ptr, g.col, g.w, g.K, g.labels)
    assert e.value.status == Bd.FW_ERR_CUDA


def test_invalid_arguments_rejected_before_device_use(libpath):
    from paper_2508_09738_gb300 import binding as Bd
    import numpy as np
    rp = np.array([0, 1, 2], np.int32)
    col = np.array([1, 0], np.int32)
    w = np.ones(2)
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(2, rp, col, w, 1, np.array([-1, -1], np.int32))
    assert e.value.status == Bd.FW_ERR_UNSUPPORTED
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(2, rp, col, w, 3, np.array([5, -1], np.int32))
    assert e.value.status == Bd.FW_ERR_INVALID_ARG
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(2, np.array([0, 2, 1], np.int32), col, w, 3, np.array([0, -1], np.int32))
    assert e.value.status == Bd.FW_ERR_GRAPH
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(2, rp, col, w, 3, np.array([0, -1], np.int32),
                         Bd.fw_seg_default_opts(class_table=7))
    assert e.value.status == Bd.FW_ERR_INVALID_ARG
    import ctypes
    f = Bd.fw_seg_forms()
    assert Bd.lib().fw_seg_get_forms(None, ctypes.byref(f)) == Bd.FW_ERR_INVALID_ARG
    graphs = [type("G", (), dict(n=2, row_ptr=rp, col=col, w=w, K=3,
                                 labels=np.array([0, -1], np.int32)))()]
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_batch_create(graphs, Bd.fw_seg_default_opts(), Bd.fw_batch_default_opts(schedule=9))
    assert e.value.status == Bd.FW_ERR_INVALID_ARG
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(2, rp, col, w, 3, np.array([0, -1], np.int32),
                         Bd.fw_seg_default_opts(eps=-1.0))
    assert e.value.status == Bd.FW_ERR_INVALID_ARG
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_seg_create(2, rp, col, w, 3, np.array([0, -1], np.int32),
                         Bd.fw_seg_default_opts(index_width=16))
    assert e.value.status == Bd.FW_ERR_INVALID_ARG


def test_large_input_size_checks_before_upload(libpath):
    """Inputs of at least 2^20 rows are uploaded before the host's planning
    pass; K outside [2, 32] is still rejected before any device call."""
    from paper_2508_09738_gb300 import binding as Bd
    import numpy as np
    n = 1 << 20
    rp = np.arange(n + 1, dtype=np.int32)          # never read beyond rp[0] and rp[n]
    col = np.zeros(n, np.int32)
    w = np.ones(n)
    lab = np.full(n, -1, np.int32)
    for K in (1, 33):
        with pytest.raises(Bd.FwError) as e:
            Bd.fw_seg_create(n, rp, col, w, K, lab)
        assert e.value.status == Bd.FW_ERR_UNSUPPORTED


def test_noalloc_energy_host_checks(libpath):
    """fw_energy_noalloc rejects sizes above its static scratch and bad
    arguments on the host, before any device pointer is touched."""
    from paper_2508_09738_gb300 import binding as Bd
    fake = 0x1000                         # never dereferenced: the checks come first
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_energy_noalloc(Bd.FW_NOALLOC_MAX_N + 1, 3, fake, fake, fake, 8, fake, 3, 0,
                             50.0, 1000.0)
    assert e.value.status == Bd.FW_ERR_UNSUPPORTED
    assert str(Bd.FW_NOALLOC_MAX_N) in str(e.value)
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_energy_noalloc(10, 1, fake, fake, fake, 8, fake, 3, 0, 50.0, 1000.0)
    assert e.value.status == Bd.FW_ERR_INVALID_ARG
    with pytest.raises(Bd.FwError) as e:
        Bd.fw_energy_noalloc(10, 3, fake, fake, fake, 8, fake, 2, 0, 50.0, 1000.0)
    assert e.value.status == Bd.FW_ERR_INVALID_ARG


def test_product_code_never_imports_oracle():
    """The CUDA path and its binding share no code with the oracle."""
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(p).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert all(not a.name.startswith("oracle") for a in node.names), p
                    if isinstance(node, ast.ImportFrom):
                        assert not (node.module or "").startswith("oracle"), p
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert "oracle/" not in open(p).read(), p


@pytest.mark.parametrize("name", ["blobs2k", "sbm200k"])
def test_product_form_weights_round_like_the_oracle(name):
    """The build kernel forms W_hat_ij as (w_ij * d_i^-1/2) * d_j^-1/2 with
    d_i^-1/2 = 1 / sqrt(d_i), all IEEE FP64 operations (so numpy reproduces
    them exactly); the oracle forms w_ij / sqrt(d_i d_j).  The FP64 values
    differ by a few ulp, and the stored FP32 / BF16 weights must not."""
    import numpy as np
    import oracle.gfw as O
    from paper_2508_09738_gb300 import workloads as W
    g = W.make_config_graph(name)
    d = O.degrees(g.n, g.row_ptr, g.col, g.w)
    ref = O.normalized_weights(g.n, g.row_ptr, g.col, g.w)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    s = 1.0 / np.sqrt(d)
    prod = (g.w * s[rows]) * s[g.col]
    assert np.max(np.abs(prod - ref) / np.spacing(ref)) <= 8
    for dt in ("f32", "bf16"):
        assert np.array_equal(O.round_weights(prod, dt), O.round_weights(ref, dt))
