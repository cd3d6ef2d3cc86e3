"""The balanced split of a fused call (host arithmetic behind the C ABI, no
GPU): every chain group must advance exactly k transitions, in order, each
launch fitting one wave of at most R CTAs of at most gpb groups; the split
is taken only where a CTA's step cost grows with its groups."""
import itertools

import pytest


@pytest.fixture(scope="module")
def P():
    from paper_1508_07828_gb300 import _build
    _build.build()
    import paper_1508_07828_gb300 as P
    return P


def _ctas(seg):
    """CTAs of one segment as (first group, groups, steps, offset): CTA b of
    nb takes groups first + b*groups/nb .. first + (b+1)*groups/nb - 1."""
    nb, g0, ng, steps, off = seg
    return [(g0 + b * ng // nb, (b + 1) * ng // nb - b * ng // nb, steps, off) for b in range(nb)]


def _check_cover(launches, G, R, gpb, k):
    done = [0] * G
    for launch in launches:
        ctas = [c for seg in launch for c in _ctas(seg)]
        assert 0 < len(ctas) <= R  # one wave
        seen = set()
        for g0, ng, steps, off in ctas:
            assert 0 <= ng <= gpb
            if ng:
                assert 1 <= steps
            for g in range(g0, g0 + ng):
                assert 0 <= g < G and g not in seen
                seen.add(g)
                assert done[g] == off  # continues where the group stopped
                done[g] += steps
    assert done == [k] * G


def test_large_workload_split(P):
    """n = 2000, 16384 chains (512 groups) on 152 SMs, 1024 threads: 96 CTAs
    of 3 groups for all steps and 56 of 4 groups for the share the step-cost
    model gives (item rounds + 1.5: 7.5 / 9.5), then the 224 lagging groups
    over all 152 SMs."""
    k = 256
    L = P.pbn_balance_phases(512, 152, 4, 1, 1024, 2000, k)
    assert L is not None
    x = int(k * 7.5 / 9.5)
    assert L[0] == [(96, 0, 288, k, 0), (56, 288, 224, x, 0)]
    assert L[1] == [(152, 288, 224, k - x, x), (0, 0, 0, 0, 0)]
    _check_cover(L, 512, 152, 4, k)


@pytest.mark.parametrize("G,R,gpb,T,threads,n,k", [
    (100, 152, 1, 1, 64, 100, 1000),     # fewer groups than SMs
    (304, 152, 2, 1, 1024, 2000, 1000),  # a whole multiple
    (512, 152, 4, 1, 1024, 2000, 63),    # too few steps
    (202, 152, 2, 1, 64, 18, 1000),      # every item in one round: no step-cost difference
    (512, 152, 3, 1, 1024, 2000, 1000),  # gpb below q + 1 (the one-launch shape takes several waves)
])
def test_one_launch_cases(P, G, R, gpb, T, threads, n, k):
    assert P.pbn_balance_phases(G, R, gpb, T, threads, n, k) is None


def test_every_split_covers_every_group_in_order(P):
    splits = 0
    for R, n, threads, T, k in itertools.product([1, 3, 7, 152], [18, 100, 600, 2000], [32, 256, 1024], [1, 2],
                                                 [64, 65, 100, 4097]):
        for G in range(R + 1, 5 * R + 2, max(1, R // 7)):
            gpb = -(-G // R)
            L = P.pbn_balance_phases(G, R, gpb, T, threads, n, k)
            if L is None:
                continue
            splits += 1
            _check_cover(L, G, R, gpb, k)
    assert splits > 100


@pytest.mark.parametrize("args", [(0, 152, 4, 1, 1024, 2000, 256), (512, 0, 4, 1, 1024, 2000, 256),
                                  (512, 152, 4, 3, 1024, 2000, 256), (512, 152, 4, 1, 1024, 2000, -1),
                                  (512, 152, 4, 1, 0, 2000, 256), (512, 152, 4, 1, 1024, 2000, (1 << 30) + 1)])
def test_invalid_arguments(P, args):
    with pytest.raises(P.PbnError) as e:
        P.pbn_balance_phases(*args)
    assert e.value.status == P.PBN_ERR_INVALID
