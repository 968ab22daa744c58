"""Shared-memory layouts of the Stockham exchanges (host-side check, no GPU).

The engine of xft_engine.cuh writes sample j of virtual thread i' of pass p to
position (i' - k) R + k + j Ns (k = i' mod Ns) of the next pass's buffer and
reads sample e of thread i from position i + e T, with one padding slot every
2^PS samples.  These tests enumerate, for every warp-wide exchange access,
the 32-bit bank of each lane's 8-byte sample and count the wavefronts per
half-warp, for
  * rows (one signal's threads consecutive, PS = 4), and
  * the interleaved columns of the 2-D kernels (G columns per CTA, lane
    c + G i), with the padding PS and column offset CO that the persistent
    column kernel k_xft_cols uses (cols_shape in k_general.cu).
"""
import pytest


def pad(p, ps):
    return p + (p >> ps)


def radices(L, LE):
    N = 1 << L
    E = (1 << LE) if L >= LE else N
    P = -(-L // LE) if L >= LE else 1
    first = 1 << (L - LE * (P - 1))
    return N, E, N // E, [first] + [1 << LE] * (P - 1)


def exchanges(L, LE, lane_map, threads, ps, base_of):
    """Yield (kind, pass, addresses of the 32 lanes) for every warp access."""
    N, E, T, rad = radices(L, LE)
    ns = 1
    for p, R in enumerate(rad):
        V = E // R
        if p < len(rad) - 1:
            for vv in range(V):
                for j in range(R):
                    for w in range(max(1, threads // 32)):
                        a = []
                        for lane in range(32):
                            sl, i = lane_map(w * 32 + lane)
                            ip = i + vv * T
                            k = ip & (ns - 1)
                            a.append(base_of(sl) + pad((ip - k) * R + k + j * ns, ps))
                        yield "store", p, a
            for e in range(E):
                for w in range(max(1, threads // 32)):
                    a = []
                    for lane in range(32):
                        sl, i = lane_map(w * 32 + lane)
                        a.append(base_of(sl) + pad(i + e * T, ps))
                    yield "load", p, a
        ns *= R


def wavefronts(addrs):
    """8-byte samples: a half-warp's 16 lanes need max over bank pairs of the
    number of distinct samples on that pair (1 = conflict-free)."""
    worst = 0
    for half in (addrs[:16], addrs[16:]):
        pairs = {}
        for x in set(half):
            pairs.setdefault(x % 16, set()).add(x)
        worst = max(worst, max(len(v) for v in pairs.values()))
    return worst


@pytest.mark.parametrize("L", [8, 9, 10, 11, 12, 13])
def test_row_exchanges_conflict_free(L):
    N, E, T, _ = radices(L, 4)
    np_ = N + (N >> 4)
    spc = max(1, 256 // T)
    threads = T * spc
    accesses = list(exchanges(L, 4, lambda t: (t // T, t % T), threads, 4,
                              lambda sl: sl * np_))
    assert accesses and all(wavefronts(a) == 1 for _, _, a in accesses)


# (L, G, PS, CO) of the persistent column kernel (cols_shape), and the
# exchanges allowed to keep a 2-way conflict
COLUMN_LAYOUTS = [
    (9, 4, 3, 4, set()),
    (10, 4, 3, 4, {("store", 0)}),
    (11, 4, 2, 4, set()),
    (12, 2, 3, 8, set()),
]


@pytest.mark.parametrize("L,G,PS,CO,two_way", COLUMN_LAYOUTS)
def test_column_exchanges(L, G, PS, CO, two_way):
    N, E, T, _ = radices(L, 3)
    strc = N + (N >> PS) + CO
    seen = {}
    for kind, p, a in exchanges(L, 3, lambda t: (t % G, t // G), T * G, PS,
                                lambda sl: sl * strc):
        seen[(kind, p)] = max(seen.get((kind, p), 0), wavefronts(a))
    for key, ways in seen.items():
        assert ways <= (2 if key in two_way else 1), (key, ways)


def test_column_padding_of_the_plain_engine_conflicts():
    """The default padding (PS = 4, columns 16/G samples apart) leaves the
    4-way conflict of the first exchange at N = 2048 that the column
    kernel's layout removes."""
    L, G = 11, 4
    N = 1 << L
    strc = N + (N >> 4) + 16 // G
    worst = max(wavefronts(a) for kind, p, a in
                exchanges(L, 3, lambda t: (t % G, t // G), (N // 8) * G, 4, lambda sl: sl * strc)
                if (kind, p) == ("store", 0))
    assert worst == 4
