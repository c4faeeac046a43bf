"""The oracle's form of Algorithm 1 (Sec. 4.1.3): its verdicts follow from the
definitions (threshold theta = p G, at most round(t (1 - p_succ)) fails), its
early exit does not change the answer, and the cases where the answer is fixed
by the parameters alone come out right."""
import numpy as np


def _inst(orc):
    # K_{4,4} ferromagnet: ground energy -16 (all +1 or all -1)
    eu, ev, col = orc.biclique_graph(4)
    return eu, ev, np.ones(eu.size), col


def test_fixed_answers(orc):
    eu, ev, J, col = _inst(orc)
    G = -16.0
    kw = dict(trials=12, beta_i=0.35, beta_f=3.5, i_max=40, seed=5)
    # p_succ = 0: every budget passes (m_max = t)
    assert orc.find_imin(eu, ev, J, None, col, G, 1.0, 0.0, 2, 2, **kw) == 2
    # theta = p G below the ground energy: no trial can pass
    assert orc.find_imin(eu, ev, J, None, col, G, 1.01, 1.0, 2, 2, **kw) is None
    # p = 0: theta = 0 and a trial fails only if its best energy is > 0; the initial
    # state counts as found, and E(m) + E(-m) = 0 at h = 0 ... best <= the initial energy,
    # so the verdict is decided by the trials' best energies, recomputed here:
    i = orc.find_imin(eu, ev, J, None, col, G, 0.0, 1.0, 2, 2, **kw)
    S = 1
    b = orc.anneal(eu, ev, J, None, col, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S), 12, 5 + 2)["best_E"]
    assert (i == 2) == bool(np.all(b <= 0.0))


def test_early_exit_gives_the_full_count_answer(orc):
    eu, ev, J, col = _inst(orc)
    rng = np.random.default_rng(3)
    J = np.where(rng.random(eu.size) < 0.5, 1.0, -1.0)
    # reference "ground": the lowest energy over a long oracle run
    G = orc.anneal(eu, ev, J, None, col, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, 200), 64, 9)["best_E"].min()
    t, p, ps, i0, di, imax, seed = 10, 1.0, 0.8, 1, 1, 12, 100
    got = orc.find_imin(eu, ev, J, None, col, G, p, ps, i0, di, trials=t, beta_i=0.35, beta_f=3.5, i_max=imax,
                        seed=seed)
    # full count without early exit
    m_max = int(np.floor(t * (1 - ps) + 0.5))
    ref = None
    for i in range(i0, imax + 1, di):
        S = (i + 1) // 2
        b = orc.anneal(eu, ev, J, None, col, orc.schedule(orc.SCHED_LINEAR, 0.35, 3.5, S), t, seed + i)["best_E"]
        if int((b > p * G).sum()) <= m_max:
            ref = i
            break
    assert got == ref
