"""The operator comparisons of Sections 6.2 and 7.2 on the GPU (Gaussian-hill workload at full
size, FP32; comparisons.py): seismogram errors of the upwind orders 2 to 7 and the traditional
operators of orders 2, 4 and 6 against an order-6 run on a mesh refined by 2.

The paper's findings tested here: at the same order the upwind operator beats the traditional
one (Section 7.2's upwind-6 against traditional-6, here also at order 4), and the error falls
with the even upwind orders 2, 4, 6."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def result():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_02600_gb300.comparisons import compare
    r = compare()
    for k, v in sorted(r["errors"].items(), key=lambda kv: (kv[0][1], kv[0][0])):
        print(f"{k[1]:>11} {k[0]}: relative L2 seismogram error {v:.4f}")
    return r


def test_upwind_beats_traditional_at_equal_order(result):
    e = result["errors"]
    assert e[(6, "upwind")] < e[(6, "traditional")]
    assert e[(4, "upwind")] < e[(4, "traditional")]


def test_even_upwind_orders_converge(result):
    e = result["errors"]
    assert e[(6, "upwind")] < e[(4, "upwind")] < e[(2, "upwind")]
