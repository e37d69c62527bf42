"""Host-side model of the single-CTA sweep's fold schedule (Eq. (13)-(14) in
blocks of 32 rows): which dx each row block receives in which step.

The kernel solves block J in step G = t*nb + J from its stored residual plus
dx_{G-1} (warp 0's partial).  Its helper warp folds dx_{G-2} (not in step 0)
and then dx_{G-1} into block J+1; its updater warps fold dx_{G-2} into every
block but J and J+1 (in step 0: only into block nb-1, which a resumed state
still lacks it in); after the last step a drain folds dx_{Gend-2} into every
block but 0 and nb-1.  The team form leaves block nb-1 through dx_{Gend-3} and
every other block through dx_{Gend-2}, and resumes from that state.

The Gauss-Seidel iteration is exact only if every block holds every dx in
step order, holds all of them through dx_{G-2} when it is solved, and ends in
the team form's state; these tests check that for many sizes, sweep counts
and both starts (zero and resumed)."""
import pytest


def run_schedule(nb, iters, resumed):
    Gend = iters * nb
    # the team form's state at the start of a call: block nb-1 through step -3,
    # the others through step -2 (a fresh start has no dx at all)
    recv = {b: ([-3] if b == nb - 1 else [-3, -2]) if resumed else [] for b in range(nb)}
    solved_with = []

    def fold(block, step):
        if step < 0 and not resumed:
            return  # dx of steps before a fresh start are zero
        recv[block].append(step)

    for G in range(Gend):
        J = G % nb
        Jp1 = (J + 1) % nb
        solved_with.append((G, J, list(recv[J])))
        if G > 0:
            fold(Jp1, G - 2)
        fold(Jp1, G - 1)
        for b in range(nb):
            if G == 0:
                if b == (J - 1) % nb:
                    fold(b, G - 2)
            elif b not in (J, Jp1):
                fold(b, G - 2)
    if Gend > 0:
        for b in range(nb):
            if b not in (0, nb - 1):
                fold(b, Gend - 2)
    return recv, solved_with


@pytest.mark.parametrize("nb", [4, 5, 7, 21, 32])
@pytest.mark.parametrize("iters", [1, 2, 5])
@pytest.mark.parametrize("resumed", [False, True])
def test_every_block_gets_every_dx_in_order(nb, iters, resumed):
    recv, solved_with = run_schedule(nb, iters, resumed)
    first = -3 if resumed else 0
    for G, J, held in solved_with:
        # stored residual current through dx_{G-2}; dx_{G-1} is warp 0's partial
        assert held == list(range(first, G - 1)), (G, J)
    Gend = nb * iters
    for b in range(nb):
        last = Gend - 3 if b == nb - 1 else Gend - 2
        assert recv[b] == list(range(first, last + 1)), b


def test_zero_sweeps_leave_the_state():
    recv, solved = run_schedule(8, 0, True)
    assert not solved
    assert recv == {b: ([-3] if b == 7 else [-3, -2]) for b in range(8)}


def test_a_dropped_fold_is_caught():
    """The checks above fail when one fold is left out (a skip set one block too wide)."""
    nb, iters = 6, 2
    Gend = nb * iters
    recv = {b: [] for b in range(nb)}
    for G in range(Gend):
        J, Jp1 = G % nb, (G + 1) % nb
        if G > 0:
            recv[Jp1].append(G - 2)
        recv[Jp1].append(G - 1)
        for b in range(nb):
            if G > 0 and b not in (J, Jp1, (J + 2) % nb):   # wrong: block J+2 left out
                recv[b].append(G - 2)
    complete = all(recv[b] == list(range(0, (Gend - 3 if b == nb - 1 else Gend - 2) + 1)) for b in range(nb))
    assert not complete


# ---- which warps run the single-CTA steps (a mismatch between the named
# barrier's thread count and the warps that reach it would stall the CTA)
SOLO_THREADS, SOLO_UPD_THREADS = 512, 352


def solo_updater(w):
    return w >= 2 and (w & 3) != 0


def solo_upd_index(w):
    return w - 2 - (w >> 2)


@pytest.mark.parametrize("S", [97, 127, 128, 129, 255, 256, 300, 657, 1023, 1024, 1280, 1281, 1408, 1409, 2000, 4096,
                               8000])
def test_step_barrier_counts_the_warps_that_reach_it(S):
    n_upd_rows = min(SOLO_UPD_THREADS // 32, (S + 127) // 128)
    n_active = 3 + n_upd_rows + (1 if n_upd_rows < SOLO_UPD_THREADS // 32 else 0)
    nwarps = SOLO_THREADS // 32
    active = [w == 0 or w == 1 or w == 4 or w == nwarps - 1 or (solo_updater(w) and solo_upd_index(w) < n_upd_rows)
              for w in range(nwarps)]
    assert sum(active) == n_active
    # every group of four rows belongs to an updater thread of an active warp,
    # and the warps left out hold no group (thread ut holds groups ut, ut + 352, ...)
    groups = (S + 3) // 4
    owner = {}
    for w in range(nwarps):
        if not solo_updater(w):
            continue
        for lane in range(32):
            ut = solo_upd_index(w) * 32 + lane
            for g in range(ut, groups, SOLO_UPD_THREADS):
                assert g not in owner
                owner[g] = w
    assert sorted(owner) == list(range(groups))
    assert all(active[w] for w in owner.values())
