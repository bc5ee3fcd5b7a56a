"""Shared-memory index bounds of the walk kernel's layout, checked on the CPU for every length.

A mirror of the layout rule (tiles of M neighbours at class indices q0 = 3 mod 4, the reversed arrays
offset by Qr = 2 mod 4, lag groups padded to multiples of M/4 + 1) and of every index the scan, the
Delta E finish, the P bookkeeping and the table update derive from it.  Any layout the rule accepts
must keep every byte-window and table access inside its array; the kernel relies on this instead of
run-time bounds checks.
"""
import pytest

# CPU check of every shared-memory index the scan / table / P code touches, for all L, modes, p, M.
kQOff, kDirBytes, kClassBytes, kCLen = 3, 1216, 608, 608

def pos_q(skew, i):
    return ((i - (1 if i & 1 else 2)) >> 1) + kQOff if skew else i - 1 + kQOff

def q_pos(skew, cls, q):
    return 2 * (q - kQOff) + (1 if cls else 2) if skew else q - kQOff + 1

def layout(L, skew, p, M, H=1):
    lam = 2 if skew else 1
    G = (L - 1) // lam; NG = (G + 3) // 4; c = (L + 1) // 2; mlast = c if skew else L
    tiles = []; qmax_end = 0
    for cls in range(2 if skew else 1):
        i_lo, i_hi = p + 1, mlast
        if skew:
            if (i_lo & 1) != cls: i_lo += 1
            if (i_hi & 1) != cls: i_hi -= 1
        if i_lo > i_hi: continue
        q_lo, q_hi = pos_q(skew, i_lo), pos_q(skew, i_hi)
        first = ((q_lo - 3) // 4) * 4 + 3
        nt = (q_hi - first + 1 + M - 1) // M
        tiles += [(cls, first + t * M) for t in range(nt)]
        qmax_end = max(qmax_end, first + nt * M - 1)
    Qr = qmax_end + ((2 - (qmax_end & 3)) & 3)
    cap = kClassBytes if skew else kDirBytes
    R = M // 4 + 1
    if H == 1:
        NGh = -(-NG // R) * R; NGend = NGh
    else:
        half = (NG + 1) // 2; NGh = -(-half // R) * R; rest = NG - NGh
        NGend = NGh + (-(-rest // R) * R if rest > 0 else 0)
    ntiles = [sum(1 for t in tiles if t[0] == cls) for cls in range(2)]
    ok = (qmax_end + 4 * NGend + 8 < cap and Qr + 4 * NGend + 8 < cap and 2 * qmax_end < cap
          and 4 * NGend <= kCLen)
    return dict(lam=lam, G=G, NG=NG, c=c, mlast=mlast, tiles=tiles, Qr=Qr, cap=cap, ok=ok, NGh=NGh, NGend=NGend, R=R,
                ntiles=ntiles, cl=kCLen, qmax_end=qmax_end, L=L, skew=skew)


def compact(ly):
    """Mirror of compact_layout: the class arrays and the table shrunk to what the length needs."""
    n_cls = (ly["L"] + 1) // 2 if ly["skew"] else ly["L"]
    need = max(ly["qmax_end"] + 4 * ly["NGend"] + 8, ly["Qr"] + 4 * ly["NGend"] + 8, 2 * ly["qmax_end"] + 1,
               kQOff + n_cls + 1)
    out = dict(ly)
    out["cap"] = -(-need // 16) * 16
    out["cl"] = -(-max(4 * ly["NGend"], ly["G"] + 1) // 8) * 8
    assert out["cap"] <= ly["cap"] and out["cl"] <= kCLen  # never larger than the fixed slab
    return out



VARIANTS = ((8, 1), (12, 1), (16, 1), (16, 2))


def _cases():
    for L in range(3, 577):
        for skew in (0, 1):
            if skew and L % 2 == 0:
                continue
            kk = (L - 1) // 2
            for p in sorted(set([0, 1, 2, 3, 24, min(kk, 100), kk if skew else L - 1])):
                if skew and p > kk:
                    continue
                if not skew and p >= L:
                    continue
                yield L, skew, p


def _check(L, skew, p, M, H, small=False):
    ly = layout(L, skew, p, M, H)
    if not ly["ok"]:
        return 0
    if small:
        ly = compact(ly)
    words = ly["cap"] // 4
    K = M // 4 + 1
    covered = set()
    c = ly["c"]
    for cls, q0 in ly["tiles"]:
        assert (q0 + 1) % 4 == 0 and (ly["Qr"] - q0 + 1) % 4 == 0
        tf0 = (q0 + 1) >> 2
        tb0 = ((ly["Qr"] - q0 + 1) >> 2) - M // 4
        idx, idxb = [], []
        for (ub, ue) in ([(0, ly["NGh"])] if H == 1 else [(0, ly["NGh"]), (ly["NGh"], ly["NGend"])]):
            idx += [tf0 + ub + a for a in range(K)] + [tf0 + ub + u + K for u in range(ue - ub)]
            idxb += [tb0 + ub + a for a in range(K)] + [tb0 + ub + u + K for u in range(ue - ub)]
        assert min(idx) >= 0 and max(idx) < words and min(idxb) >= 0 and max(idxb) < words, (L, skew, p, M, q0)
        for j in range(M):
            q = q0 + j
            m = q_pos(skew, cls, q)
            if p + 1 <= m <= ly["mlast"]:
                covered.add(m)
            # finish / table update: windows s_{m +- lambda g} for g = 1..G and the neighbour itself
            for g in (1, ly["G"]):
                assert 0 <= q + g < ly["cap"] and 0 <= ly["Qr"] - q + g < ly["cap"], (L, skew, p, M, q, g)
            assert 0 <= q < ly["cap"] and 0 <= ly["Qr"] - q < ly["cap"]
            # table update: realigned words (q + 1) / 4 + u and (Qr - q + 1) / 4 + u, + 1, for u < NG
            assert (q + 1) // 4 + ly["NG"] < words and (ly["Qr"] - q + 1) // 4 + ly["NG"] < words
            # P bookkeeping: class index max(2q - q_f, 0) for every flipped position f of this class; the
            # largest index comes from the smallest q_f (flipped positions lie in p+1..mlast)
            f_lo = p + 1 + (1 if skew and ((p + 1) & 1) != cls else 0)
            if f_lo <= ly["mlast"]:
                assert max(2 * q - pos_q(skew, f_lo), 0) < ly["cap"], (L, skew, p, M, q)
    if skew:
        for f in range(p + 1, c):  # the mirror L + 1 - f of a pair flip: class index c + 6 - b - q_f
            b = 1 if f & 1 else 2
            assert pos_q(skew, L + 1 - f) == c + 6 - b - pos_q(skew, f)
            # the pair term reads C16[c - f - 1]; a slot without one reads C16[cl - 1], which lies beyond
            # G (always zero)
            assert 0 <= c - f - 1 < ly["cl"]
        assert ly["cl"] - 1 >= ly["G"]
    # the table arrays: entries 0..4 NG - 1 are rewritten by the update, 4 NGend are read by the scan
    assert 4 * ly["NGend"] <= ly["cl"] and 4 * ly["NG"] <= ly["cl"]
    assert covered == set(range(p + 1, ly["mlast"] + 1)), (L, skew, p, M)
    return 1


@pytest.mark.parametrize("small", [False, True])
@pytest.mark.parametrize("M,H", VARIANTS)
def test_layout_indices_stay_inside_their_arrays(M, H, small):
    """Fixed slabs (every length up to 576) and slabs shrunk to the length (the walk kernels' dynamic
    shared memory): every index inside its array."""
    tested = sum(_check(L, skew, p, M, H, small) for L, skew, p in _cases())
    assert tested > 1000


def test_every_length_fits_some_variant():
    for L in range(3, 577):
        for skew in ((0, 1) if L % 2 else (0,)):
            assert any(layout(L, skew, 0, M, H)["ok"] for M, H in VARIANTS), (L, skew)


def test_fold_entry_split_without_divide():
    """The P fold gives group lane n (0..GL-1, GL = 16 or 32) its first (slot k, task tl) of a class as
    k = (n * magic) >> 16, tl = n - k * tasks, and steps by the same split of GL, with magic =
    ceil(2^16 / tasks): that must be n // tasks for every n <= 32, every class of every accepted layout."""
    seen = 0
    for M, H in VARIANTS:
        for L, skew, p in _cases():
            ly = layout(L, skew, p, M, H)
            if not ly["ok"]:
                continue
            for n in ly["ntiles"]:
                nt = n * H
                if nt == 0:
                    continue
                magic = ((1 << 16) + nt - 1) // nt
                assert all((e * magic) >> 16 == e // nt for e in range(33)), (L, skew, p, M, H, nt)
                seen += 1
    assert seen > 1000


def _window_bytes(bits, L, p, d, rev):
    """Mirror of the device construction of one byte-window word: positions p, p+d, p+2d, p+3d."""
    plast = p + 3 * d
    if p > L or plast < 1:
        return 0x01010101
    b = p - 1
    x = (bits >> b) if b >= 0 else (bits << (-b))
    if d == 2:
        x &= 0x55
        x = (x | (x >> 1)) & 0x33
        x = (x | (x >> 2)) & 0x0F
    else:
        x &= 0xF
    lo = (1 - p + d - 1) // d if p < 1 else 0
    hi = (plast - L + d - 1) // d if plast > L else 0
    v = ((0xF << lo) & (0xF >> hi)) & 0xF
    xv, pad = x & v, v ^ 0xF
    if rev:
        xv = int('{:04b}'.format(xv)[::-1], 2)
        pad = int('{:04b}'.format(pad)[::-1], 2)
    spread = lambda n: (n * 0x204081) & 0x01010101  # bit e -> bit 8e, no carries
    return 2 * spread(xv) + spread(pad)


def test_byte_windows_four_positions_per_word():
    """Every word of the forward and reversed byte windows, built four positions at a time from the bits
    (one shift, every other bit for the skew classes, a multiply spreading 4 bits to 4 bytes, the pads),
    equals the per-byte definition: s + 1 inside 1..L, 1 outside."""
    import random
    rng = random.Random(5)
    checked = 0
    for L in list(range(3, 100)) + [449, 450, 451, 527, 575, 576]:
        for skew in (0, 1):
            if skew and L % 2 == 0:
                continue
            ly = layout(L, skew, min(24, (L - 1) // 2) if skew else 0, 16, 2)
            if not ly["ok"]:
                continue
            bits = rng.getrandbits(L)
            lam = 2 if skew else 1
            byte = lambda i: (2 if (bits >> (i - 1)) & 1 else 0) if 1 <= i <= L else 1
            words = compact(ly)["cap"] // 4
            for cls in range(2 if skew else 1):
                first = q_pos(skew, cls, kQOff)
                for w in range(words):
                    f = _window_bytes(bits, L, first + lam * (4 * w - kQOff), lam, False)
                    assert f == sum(byte(q_pos(skew, cls, 4 * w + e)) << (8 * e) for e in range(4)), (L, skew, cls, w)
                    r = _window_bytes(bits, L, first + lam * (ly["Qr"] - 4 * w - 3 - kQOff), lam, True)
                    assert r == sum(byte(q_pos(skew, cls, ly["Qr"] - 4 * w - e)) << (8 * e) for e in range(4)), (L, skew, cls, w)
                    checked += 1
    assert checked > 5000
