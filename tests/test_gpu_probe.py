"""The solver's team plan query and the hand-over latency probe (measurement aids)."""
import math

import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1608_05179_gb300")
D = P.damas


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = D.Context(0)
    yield c
    c.close()


def test_solve_plan(ctx):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for S in (1, 32, 33, 657, 6561, 25921):
        for dt in (D.F32, D.BF16):
            n, R, res = D.damas_solve_plan(ctx, S, dt)
            nb = -(-S // 32)
            assert R % 32 == 0 and n * R >= nb * 32 and (n - 1) * R < nb * 32
            assert 1 <= n <= max(1, sms)
    # the compressed 81x81 system runs on one CTA (no hand-overs); asked to keep A in
    # shared memory, it takes a resident team; the full grid streams A
    assert D.damas_solve_plan(ctx, 657, D.F32) == (1, 672, False)
    n, R, res = D.damas_solve_plan(ctx, 657, D.F32, a_placement=D.PLACE_RESIDENT)
    assert res and n > 1
    assert not D.damas_solve_plan(ctx, 6561, D.F32)[2] and D.damas_solve_plan(ctx, 6561, D.F32)[0] > 1
    # forced team sizes and placements are honoured
    assert D.damas_solve_plan(ctx, 657, D.F32, ctas=21, a_placement=D.PLACE_STREAM) == (21, 32, False)
    n, R, res = D.damas_solve_plan(ctx, 657, D.F32, a_placement=D.PLACE_STREAM)
    assert not res


def test_handover_probe(ctx):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ns = D.damas_handover_probe(ctx, rounds=50)
    assert len(ns) == sms - 1
    assert all(math.isfinite(v) and 10.0 < v < 100000.0 for v in ns)
    print(f"hand-over one-way ns: min {min(ns):.0f} median {sorted(ns)[len(ns) // 2]:.0f} max {max(ns):.0f}")
    assert len(D.damas_handover_probe(ctx, rounds=5, max_pairs=3)) == 3


def test_handover_probe_bounded_wait(ctx):
    """A wait bound of 1 us runs out (CTA 1 waits for its turn far longer): the
    call reports DAMAS_ETIMEDOUT and the context keeps working."""
    with pytest.raises(D.DamasError) as ei:
        D.damas_handover_probe(ctx, rounds=50, max_pairs=8, timeout_us=1)
    assert ei.value.code == P._lib.DAMAS_ETIMEDOUT
    assert len(D.damas_handover_probe(ctx, rounds=10, max_pairs=2)) == 2
