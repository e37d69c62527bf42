"""Host logic of band processing (§6): how the bins of a band share the CTAs of
one persistent launch.  No GPU is needed."""
import pytest

B = pytest.importorskip("paper_1608_05179_gb300.band")


def test_balanced_team_sizes():
    """Balanced plans fit the capacity, give every bin at least one CTA and at
    most one per 32-row block, favour the long chains, and leave the estimated
    times of the bins that received extra CTAs within one CTA's worth of each other."""
    S_f = [600, 1200, 9000, 14641, 3000, 64, 33]
    for cap, r0 in [(304, 512.0), (152, 256.0), (40, 1024.0), (7, 512.0)]:
        P = B.team_sizes_balanced(S_f, cap, r0)
        nb = [-(-s // 32) for s in S_f]
        assert sum(P) <= max(cap, len(S_f)) and all(1 <= p <= n for p, n in zip(P, nb))
        assert P[3] >= P[2] >= P[4] >= P[1] >= P[0]
        cost = [n * (1 + s / p / r0) for n, s, p in zip(nb, S_f, P)]
        grown = [f for f in range(len(S_f)) if 1 < P[f] < nb[f]]
        if grown:
            worst = max(cost)
            for f in grown:
                before = nb[f] * (1 + S_f[f] / (P[f] - 1) / r0)
                assert before >= worst - 1e-9 or cost[f] == worst


def test_team_sizes_fit_capacity():
    S_f = [600, 1200, 9000, 14641, 3000]
    P = B.team_sizes(S_f, 512, 148)
    assert sum(P) <= 148 and all(p >= 1 for p in P)
    P2 = B.team_sizes(S_f, 512, 10)
    assert sum(P2) <= max(10, len(S_f)) and P2[3] >= P2[0]
