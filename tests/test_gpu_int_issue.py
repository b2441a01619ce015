"""Integer-issue microbenchmark (pt_int_issue_rate): every kind runs, its time
grows in proportion to the loop count (the work is not folded away), and no
kind reports more than the SMs can issue (one warp instruction per
sub-partition per clock: 128 lane operations per SM per clock at the
highest SM clock, 2.07 GHz)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1605_03607_gb300 as pkg
    from paper_1605_03607_gb300 import build as b
    b.build()
    pkg.load()
    return pkg


@pytest.mark.parametrize("kind", ["lop3", "imad", "lop3_imad", "dp4a", "philox_round"])
def test_rate_is_bounded_and_work_scales(P, kind):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_bound = sms * 128 * 2.07e9
    ops_a, ms_a = P.int_issue_rate(kind, iters=1 << 14, reps=3)
    ops_b, ms_b = P.int_issue_rate(kind, iters=1 << 16, reps=3)
    assert ops_a > 0 and ms_a > 0 and ops_b > 0 and ms_b > 0
    assert 2.8 < ms_b / ms_a < 5.0, (ms_a, ms_b)
    assert ops_b <= 1.05 * issue_bound, (ops_b, issue_bound)


def test_rejects_bad_kind_on_gpu(P):
    with pytest.raises(P.PTError):
        P.int_issue_rate(7)
