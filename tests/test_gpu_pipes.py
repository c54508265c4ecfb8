"""The integer-pipe rate kernels (roofline denominators) run and give rates within the
SM's issue capacity: 4 sub-partitions x 32 lanes = 128 lane-operations per SM per clock."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_within_the_issue_capacity():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_6082_gb300 import build, pipes
    build.build_pipes()
    r = pipes.all_rates()
    for op in pipes.OPS:
        assert r[op] > 0, (op, r)
    for op in ("lop3", "lop3_2r", "imad_lo", "imad_lo_1r", "imad_hi", "imad_wide", "iadd3",
               "mix_imad_lo_lop3", "mix_light", "mix_imad_wide_lop3"):
        assert r[op] <= 130.0, (op, r)
    # a Philox block is 20 widening products: it cannot beat the widening-multiply rate by much
    assert r["philox_products"] <= 1.1 * r["imad_wide"], r
