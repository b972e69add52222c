"""The integer-pipe microbenchmark behind the roofline's measured peak:
it runs, reports a rate within the pipe's possible range, and refuses bad
arguments on the host."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    from paper_1910_03936_gb300 import build
    build.build()
    import paper_1910_03936_gb300 as m
    return m


def test_peak_int_runs_and_is_plausible(pf):
    import torch
    ctx = pf.pf_create(0)
    try:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for kind in (0, 1):
            ops, ms = pf.pf_peak_int(ctx, kind, 2)
            # at most 64 lanes per clock per SM at 2.5 GHz; at least a tenth of it
            ceiling = sms * 64 * 2.5e9
            assert 0.02 * ceiling < ops < ceiling, (kind, ops)
            assert ms > 0
        for bad in ((2, 1), (-1, 1), (0, 0), (0, 1001)):
            with pytest.raises(pf.PFError) as ei:
                pf.pf_peak_int(ctx, *bad)
            assert ei.value.status == 1
    finally:
        pf.pf_destroy(ctx)
