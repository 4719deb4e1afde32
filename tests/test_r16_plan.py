"""The radix-16 transform plan of the FP32 fine sweep (csrc/spectral16.cuh),
modelled on the CPU: its lane layout, butterfly positions, warp assignment and
stage order, restated here from the kernel's description (not shared with it).

- The split of a butterfly's positions by linearity of the layout over GF(2)
  equals the layout applied term by term, and every position stays in the lane.
- Every half-warp access of the plan (span-N butterflies, the warp-grouped
  span-N/16 butterflies, the middle stage, the mode packing) is checked for
  shared-memory bank conflicts by simulation (8-byte elements, 16 bank pairs).
- The warp-grouped stages and the middle stage of one warp touch the same
  (lane, point) set, so synchronising the warp alone between them is enough.
- The whole plan -- inverse stages with the 2/3-rule inputs left unread (NaN),
  the middle stage with the products, forward stages with the unread outputs
  dropped -- gives the spectra of the nonlinear products that numpy's FFT gives,
  on every bin an unpack reads."""
import numpy as np
import pytest


def pidx16(i):
    return i ^ ((i >> 4) & 15)


def positions(base, e):
    sb = pidx16(base)
    return [((sb ^ ((q * e >> 4) & 15)) + q * e) if e >= 16 else (sb ^ pidx16(q * e)) for q in range(16)]


def items(n, logl, grouped):
    """(thread, lane, j, base) of every butterfly of the span-2^logl stage."""
    nb, e = n // 16, 1 << (logl - 4)
    out = []
    for item in range(2 * nb):
        lane = (item >> 4) & 1 if grouped else item // nb
        bidx = ((item >> 5) << 4) | (item & 15) if grouped else item - lane * nb
        j = bidx & (e - 1)
        out.append((item, lane, j, ((bidx >> (logl - 4)) << logl) + j))
    return out


def conflict_degree(addrs):
    """Worst bank-pair conflict over the two half-warps of one warp access (None = inactive)."""
    worst = 1
    for h in (0, 16):
        banks = {}
        for a in addrs[h:h + 16]:
            if a is not None:
                banks.setdefault(a % 16, set()).add(a)
        worst = max([worst] + [len(v) for v in banks.values()])
    return worst


@pytest.mark.parametrize("logn", [9, 10, 11])
def test_positions_split_by_linearity(logn):
    n = 1 << logn
    for logl in (logn, logn - 4):
        e = 1 << (logl - 4)
        for _, _, _, base in items(n, logl, logl != logn):
            at = positions(base, e)
            assert at == [pidx16(base + q * e) for q in range(16)]
            assert all(0 <= a < n for a in at)
    assert sorted(pidx16(i) for i in range(n)) == list(range(n))


@pytest.mark.parametrize("logn", [9, 10, 11])
def test_plan_accesses_are_bank_conflict_free(logn):
    n, block = 1 << logn, (1 << logn) // 8
    r = 1 << (logn % 4)
    for logl, grouped in ((logn, False), (logn - 4, True)):
        its = items(n, logl, grouped)
        for w in range(block // 32):
            for q in range(16):
                addrs = [lane * 1_000_000 + positions(base, 1 << (logl - 4))[q]
                         for _, lane, _, base in its[32 * w:32 * w + 32]]
                assert conflict_degree(addrs) == 1, (logl, w, q)
    for w in range(block // 32):                     # middle stage: warp w's items, R points each
        t = np.arange(32)
        for rr in range(8 // r):
            i = (256 // r) * w + t + 32 * rr
            for q in range(r):
                assert conflict_degree([pidx16(r * int(x)) ^ q for x in i]) == 1
    k_max = (n - 1) // 3                               # mode packing: bins k and N-k, k = t + r*block
    worst = 1
    for rr in range(3):
        for w in range(block // 32):
            for neg in (0, 1):
                ks = [t + rr * block + 32 * w for t in range(32)]
                addrs = [None if (k > k_max or k == 0) else pidx16(n - k if neg else k) for k in ks]
                worst = max(worst, conflict_degree(addrs))
    assert worst <= 2   # the N-k bins of a half-warp straddle one 16-element block


@pytest.mark.parametrize("logn", [9, 10, 11])
def test_warp_owns_its_middle_section(logn):
    n, block, r = 1 << logn, (1 << logn) // 8, 1 << (logn % 4)
    e = (n // 16) // 16
    its = items(n, logn - 4, True)
    for w in range(block // 32):
        stage = {(lane, p) for _, lane, _, base in its[32 * w:32 * w + 32] for p in positions(base, e)}
        middle = set()
        for t in range(32):
            for rr in range(8 // r):
                i = (256 // r) * w + t + 32 * rr
                for q in range(r):
                    middle |= {(0, pidx16(r * i) ^ q), (1, pidx16(r * i) ^ q)}
        assert stage == middle and len(stage) == 512


def dft(x, sign):
    m = len(x)
    k = np.arange(m)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / m) @ x


def twiddles(logn):
    tab, l = {}, logn
    while l > logn % 4:
        big_l, e = 1 << l, (1 << l) // 16
        tab[l] = np.array([np.exp(-2j * np.pi * q * j / big_l) for q in range(1, 16) for j in range(e)])
        l -= 4
    return tab


def stage(z, n, sign, dif, logl, tw, prune, grouped):
    e = 1 << (logl - 4)
    for _, lane, j, base in items(n, logl, grouped):
        at = positions(base, e)
        x = np.array([0 if (prune == 1 and 6 <= q <= 9) else z[lane][at[q]] for q in range(16)], complex)
        if not dif and j:
            x[1:] *= tw[[(q - 1) * e + j for q in range(1, 16)]]
        x = dft(x, sign)
        if dif and j:
            x[1:] *= np.conj(tw[[(q - 1) * e + j for q in range(1, 16)]])
        for q in range(16):
            z[lane][at[q]] = np.nan if (prune == 2 and q >= 6 and (lane == 1 or q <= 9)) else x[q]


@pytest.mark.parametrize("logn", [9, 10])
def test_plan_computes_the_products_spectra(logn):
    n, k_max = 1 << logn, ((1 << logn) - 1) // 3
    rng = np.random.default_rng(logn)

    def field():
        c = np.zeros(n, complex)
        c[:k_max + 1] = rng.standard_normal(k_max + 1) + 1j * rng.standard_normal(k_max + 1)
        c[0] = c[0].real
        c[n - k_max:] = np.conj(c[1:k_max + 1][::-1])
        return np.fft.ifft(c).real * n

    v1, h, v2 = field(), field(), field()
    k = np.fft.fftfreq(n, 1.0 / n)
    v1x, v2x = (np.fft.ifft(1j * k * np.fft.fft(f)).real for f in (v1, v2))
    s0, s1 = np.fft.fft(v1 + 1j * h) / n, np.fft.fft(v1x + 1j * v2x) / n
    z = [np.full(n, np.nan, complex), np.full(n, np.nan, complex)]
    for b in range(n):
        if not 3 * n // 8 <= b < 5 * n // 8:       # the 2/3 rule's zero bins are never written
            z[0][pidx16(b)], z[1][pidx16(b)] = s0[b], s1[b]
    tw, r = twiddles(logn), 1 << (logn % 4)
    stage(z, n, +1, True, logn, tw[logn], 1, False)
    stage(z, n, +1, True, logn - 4, tw[logn - 4], 0, True)
    for i in range(n // r):
        p0 = pidx16(r * i)
        a, b = dft(np.array([z[0][p0 ^ q] for q in range(r)]), +1), dft(np.array([z[1][p0 ^ q] for q in range(r)]), +1)
        a, b = -a.real * b.real - 1j * a.real * b.imag, -a.imag * a.real + 0j
        a, b = dft(a, -1), dft(b, -1)
        for q in range(r):
            z[0][p0 ^ q], z[1][p0 ^ q] = a[q], b[q]
    stage(z, n, -1, False, logn - 4, tw[logn - 4], 0, True)
    stage(z, n, -1, False, logn, tw[logn], 2, False)
    p0_ref, p1_ref = np.fft.fft(-v1 * v1x - 1j * v1 * v2x), np.fft.fft(-h * v1 + 0j)
    scale = np.abs(p0_ref).max()
    read0 = list(range(k_max + 1)) + list(range(n - k_max, n))
    assert max(abs(z[0][pidx16(b)] - p0_ref[b]) for b in read0) <= 1e-12 * scale
    assert max(abs(z[1][pidx16(b)] - p1_ref[b]) for b in range(k_max + 1)) <= 1e-12 * scale
