"""The integer-pipe throughput probe behind the benchmark's ALU roofline
(paper_2010_03090_gb300/probe/alu_probe.cu): its rates are physically
plausible for a GB300 SM, so the roofline's denominator is a measurement and
not an artefact.  Needs a GPU (-m gpu)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_probe_rates_are_plausible():
    import bench
    res = bench.alu_probe(float(bench.measured_peaks().get("sm_max_mhz") or 2070.0),
                          iters=4000)
    assert "error" not in res, res
    # an SM issues at most 4 x 32 thread instructions per clock; one pipe is
    # a fraction of that, and the two pipes together more than one alone
    for op in ("lop3", "prmt", "shf", "imad"):
        assert 16.0 <= res[op] <= 130.0, (op, res)
    assert res["prmt+imad"] > 1.3 * max(res["prmt"], res["imad"]) or res["prmt+imad"] > 100, res
