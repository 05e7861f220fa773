"""Pass B with the class table in shared memory (k_passB_tab) against the
direct pass-B kernels: the same iterates, labels and statistics bit for bit
(GPU).  The table form forms every 256-row tile's total in the order of the
direct kernels, so any difference here is a bug, not rounding."""
import numpy as np
import pytest

from paper_2508_09738_gb300 import binding as B
from paper_2508_09738_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_09738_gb300 import build
    build.build()


def run(g, table, **kw):
    with B.Segmenter(g, class_table=table, iters_per_launch=16, **kw) as s:
        f = s.forms()
        st = s.solve()
        return f, s.U(), s.labels(), (st.iters, st.status, st.gap, st.objective, st.q,
                                      st.alpha, st.active_rows)


def assert_same(a, b):
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


# (K, lanes, weights, rows per class): ragged last tiles; the larger problems
# have more tiles than SMs, so blocks take runs of 2-3 tiles
CASES = [(3, 1, "f32", 1013), (4, 2, "f32", 1013), (5, 2, "bf16", 8011), (8, 4, "bf16", 1013),
         (10, 2, "f32", 9999), (10, 2, "bf16", 9999), (12, 1, "f32", 3001), (16, 4, "f32", 2003),
         (16, 2, "f32", 5003)]


@pytest.mark.parametrize("K,lanes,weights,m", CASES)
def test_class_table_equals_direct(K, lanes, weights, m):
    g = W.sbm(n=m * K, K=K, deg_in=18.0, deg_out=3.0, label_frac=0.02, seed=100 + K + m)
    kw = dict(weight_dtype=weights, lanes_per_row=lanes, max_iters=80)
    on = run(g, "on", **kw)
    off = run(g, "off", **kw)
    assert on[0].class_table == 1 and on[0].table_blocks > 0 and on[0].lanes_per_row == lanes
    assert off[0].class_table == 0 and off[0].table_blocks == 0
    # graphs of fewer than 2^15 rows store 16-bit column offsets, the rest 32-bit indices
    assert on[0].index_width == (16 if g.n <= 1 << 15 else 32)
    assert_same(on, off)


def test_class_table_auto_on_sbm200k_full_size():
    """The SBM workload (200,000 rows, K = 10, scattered columns) takes the
    table form by default; 500 iterations give the direct form's bits."""
    g = W.make_config_graph("sbm200k")
    c = W.CONFIGS["sbm200k"]
    kw = dict(weight_dtype="f32", max_iters=c["iters"], eps=c["eps"], omega0=c["omega0"])
    auto = run(g, "auto", **kw)
    off = run(g, "off", **kw)
    assert auto[0].class_table == 1 and auto[0].lanes_per_row == 2 and auto[0].kmax == 10
    assert off[0].class_table == 0
    assert auto[3][0] == c["iters"]
    assert_same(auto, off)


def test_class_table_only_where_it_applies():
    """Banded graphs stay on the direct form under auto (their class gathers
    hit L1), but may be forced onto the table; an FP64 iterate, K > 16 and a
    class array larger than shared memory keep the direct form even when it
    is asked for."""
    img = W.voronoi_image(side=300, height=211, K=4, label_frac=0.01, seed=5)
    kw = dict(max_iters=60, omega0=1e5)
    auto = run(img, "auto", **kw)
    on = run(img, "on", **kw)
    assert auto[0].index_width == 16 and auto[0].class_table == 0
    assert on[0].class_table == 1
    assert_same(auto, on)
    sb = W.sbm(n=20 * 1000, K=20, deg_in=12.0, deg_out=2.0, seed=3)
    assert run(sb, "on", max_iters=5)[0].class_table == 0            # K > 16: no 4-bit classes
    sb4 = W.sbm(n=4 * 2000, K=4, deg_in=12.0, deg_out=2.0, seed=4)
    assert run(sb4, "on", max_iters=5, weight_dtype="f64")[0].class_table == 0
    big = W.voronoi_image(side=1024, K=4, label_frac=0.01, seed=6)   # 2^20 rows: 512 KB table
    assert run(big, "on", max_iters=2, omega0=1e5)[0].class_table == 0
