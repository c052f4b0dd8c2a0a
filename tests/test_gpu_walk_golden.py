"""The GPU tree walk on the hand-built case of
tests/golden/walk_open_example.json (Eq. 1 per walk group and the r_cut
skip, every decision derived by hand): group A's interaction list has the
hand-derived length, every group's list has the oracle's length, and the
short-range force on A's particles is the pair sum over the hand-derived list
(FP64 1e-9, FP32 1e-4 of |g| + 1e-3 rms)."""
import numpy as np
import pytest

import oracle as O
import walk_golden as W
from test_oracle_walk_golden import group_of_a, hand_list_force, sorted_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def run(dzs, precision):
    cs, P, u, k, names = sorted_case()
    n = u.shape[1]
    st = dict(u=u, p=np.zeros((3, n)), g=np.zeros((3, n)), k=k, id=np.arange(n, dtype=np.uint32),
              fl=np.zeros(n, np.uint8))
    with dzs.Context(**cs["params"], precision=precision) as ctx:
        ctx.set_state(st, 0)
        g = ctx.accel(dzs.ACC_TREE)
        first, cnt, ln = ctx.walk_lists()
        wc = ctx.walk_counters()
    return cs, P, u, k, names, g, (first, cnt, ln), wc


@pytest.mark.parametrize("precision", [1, 0])
def test_gpu_walk_lists_match_the_hand_derivation(dzs, precision):
    cs, P, u, k, names, g, (first, cnt, ln), wc = run(dzs, precision)
    _, s, c = group_of_a(P, u, names)
    a = [i for i in range(len(first)) if first[i] == s and cnt[i] == c]
    assert len(a) == 1
    assert ln[a[0]] == cs["expected_list_length_A"]
    # every group: the oracle's list length
    starts, counts = O.groups(P, u)
    assert sorted(zip(first.tolist(), cnt.tolist())) == sorted(zip(starts.tolist(), counts.tolist()))
    by_first = dict(zip(first.tolist(), ln.tolist()))
    for gi, st0 in enumerate(starts.tolist()):
        assert by_first[st0] == O.interaction_count(P, u, k, group_index=gi), gi
    assert wc[0] == O.interaction_count(P, u, k)
    assert 0 < wc[1] < wc[0]


@pytest.mark.parametrize("precision", [1, 0])
def test_gpu_walk_force_is_the_hand_list_sum(dzs, precision):
    cs, P, u, k, names, g, _, _ = run(dzs, precision)
    _, s, c = group_of_a(P, u, names)
    want = np.stack([hand_list_force(cs, P, u, k, names, i) for i in range(s, s + c)], axis=1)
    got = g[:, s:s + c]
    err = np.linalg.norm(got - want, axis=0)
    ref = np.linalg.norm(want, axis=0)
    rel = err / (ref + 1e-3 * np.sqrt((ref ** 2).mean()))
    assert rel.max() <= (1e-9 if precision == 1 else 1e-4), rel.max()
