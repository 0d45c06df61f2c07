"""The range query's output placement restated in Python (host logic, no GPU):
for one warp batch and band, the band's reservation [base, base + T + nfe) must
receive every core element and every accepted fringe candidate exactly once.

- Core pieces, lane-major: lane L owns sorted positions [c0_L, c0_L + nc_L).
  Step t < min(nc) writes element t of every lane at 32 t + L; past it the lanes
  that still have an element are ranked by a ballot, at a running offset.
- Fringe stream: 32 candidates per step, lane j of step s deciding stream element
  32 s + j; an accepted candidate goes to T + (accepted before the step) + (rank
  among the step's accepted lanes) -- both when it is kept in shared memory
  during the decisions and when the decision bits are replayed.
Planted mistakes (a missing ballot rank, an off-by-one prefix) must fail."""
import numpy as np
import pytest


def popc(x):
    return bin(x).count("1")


def core_positions(nc, rank_tail=True, prefix_off=0):
    """{(lane, t): output offset} of the lane-major core writer."""
    mn, mx = min(nc), max(nc)
    out = {}
    for t in range(mn):
        for lane in range(32):
            out[(lane, t)] = 32 * t + lane + prefix_off
    pos = 32 * mn
    for t in range(mn, mx):
        m = sum(1 << lane for lane in range(32) if t < nc[lane])
        for lane in range(32):
            if t < nc[lane]:
                lt = (1 << lane) - 1
                out[(lane, t)] = pos + (popc(m & lt) if rank_tail else 0)
        pos += popc(m)
    return out


def fringe_positions(decisions, T, kept_cap=128):
    """Offsets of the accepted stream elements: from the kept pairs (at < cap)
    and from the replay of the decision bits; both as the kernel computes them."""
    F = len(decisions)
    kept, replay = {}, {}
    nfe = 0
    words = []
    for jw in range(0, F, 32):
        word = sum(1 << l for l in range(32) if jw + l < F and decisions[jw + l])
        words.append(word)
        for l in range(32):
            if (word >> l) & 1:
                at = nfe + popc(word & ((1 << l) - 1))
                if at < kept_cap:
                    kept[jw + l] = T + at
        nfe += popc(word)
    pos = T
    for s, word in enumerate(words):
        for l in range(32):
            if (word >> l) & 1:
                replay[32 * s + l] = pos + popc(word & ((1 << l) - 1))
        pos += popc(word)
    return nfe, kept, replay


CORE_CASES = [
    [0] * 32,
    [5] * 32,
    list(range(32)),
    [0] * 31 + [300],
    [1] + [40] * 31,
]


@pytest.mark.parametrize("case", range(len(CORE_CASES) + 20))
def test_core_writer_covers_the_reservation_once(case):
    rng = np.random.default_rng(case)
    nc = CORE_CASES[case] if case < len(CORE_CASES) else [int(x) for x in rng.integers(0, 60, 32)]
    if case >= len(CORE_CASES) and case % 3 == 0:
        nc[int(rng.integers(32))] = 0  # an inactive lane: no prefix at all
    out = core_positions(nc)
    T = sum(nc)
    assert len(out) == T
    assert sorted(out.values()) == list(range(T))
    # each lane's elements keep their order
    for lane in range(32):
        ps = [out[(lane, t)] for t in range(nc[lane])]
        assert ps == sorted(ps)


def test_core_writer_checks_catch_planted_mistakes():
    nc = [3] * 16 + [7] * 16
    bad = core_positions(nc, rank_tail=False)
    assert sorted(bad.values()) != list(range(sum(nc)))
    bad = core_positions(nc, prefix_off=1)
    assert sorted(bad.values()) != list(range(sum(nc)))


@pytest.mark.parametrize("F,p,T", [(0, 0.5, 0), (1, 1.0, 7), (31, 0.5, 3), (32, 1.0, 0), (137, 0.55, 900),
                                   (600, 0.6, 50), (2048, 0.3, 11), (300, 0.9, 0)])
def test_fringe_edges_follow_the_stream_in_both_paths(F, p, T):
    rng = np.random.default_rng(F + T)
    dec = (rng.random(F) < p).tolist()
    nfe, kept, replay = fringe_positions(dec, T)
    assert nfe == sum(dec)
    assert sorted(replay.values()) == list(range(T, T + nfe))
    # accepted candidates in stream order occupy consecutive slots
    acc = [j for j in range(F) if dec[j]]
    assert [replay[j] for j in acc] == list(range(T, T + nfe))
    # the kept pairs hold the first min(nfe, cap) of them at the same slots, so
    # the copy from shared memory (used when nfe <= cap) equals the replay
    assert kept == {j: replay[j] for j in acc[:128]}
    if nfe <= 128:
        assert kept == replay


def test_fringe_checks_catch_a_planted_mistake():
    dec = [True, False, True, True] * 20
    nfe, kept, replay = fringe_positions(dec, 5)
    shifted = {j: v + 1 for j, v in replay.items()}
    assert sorted(shifted.values()) != list(range(5, 5 + nfe))
