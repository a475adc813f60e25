"""Host-side checks of the FFT index tables the kernels take as constants (no GPU).

- Radix-16 column pass (`kGeoR16_8`, `kGeoR16_16` in geo_table.h): each swizzle is a
  bijection on the positions of a column, and every shared-memory access pattern of the
  pass -- the leading stage's points t + e L/16, the middle radix-16 stages, and the
  stride-1 stage's digit-reversed groups -- is free of bank conflicts (8-byte elements by
  half-warps, 16-byte elements by quarter-warps); the digit-reversed position of frequency
  t + q L/16 is that of t plus q, which the in-register spectrum multiply relies on.
- Stage twiddle tables: the radix-16 offsets (`Fft16::tw_off`) and the FP64 power-table
  offsets (`FftC::pow_off`) address the entries the table kernels write, within the
  2^m entries reserved per length.
- A step-by-step FP64 model of the radix-16 column pass (its 4 x 4 16-point DFT, stage
  order, tables and swizzled positions) forms the zero-padded circular convolution that
  numpy's FFT gives, for every leading-stage radix.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEO = os.path.join(ROOT, "paper_1612_08395_gb300", "csrc", "geo_table.h")


def geo_rows(name):
    src = open(GEO).read()
    m = re.search(name + r"\[\d+\]\s*=\s*\{(.*?)\};", src, re.S)
    assert m, name
    return [tuple(int(x) for x in g.split(",")) for g in re.findall(r"\{\s*([\d,\s]+?)\s*\}", m.group(1))]


def sw(p, prm, es):
    a, b, c, d = prm
    if es == 8:
        return p ^ ((((p >> a) ^ (p >> b)) & 7) | ((((p >> c) ^ (p >> d)) & 1) << 3))
    return p ^ ((((p >> a) ^ (p >> b)) & 3) | ((((p >> c) ^ (p >> d)) & 1) << 2))


def radices16(logL):
    rb = logL & 3
    return ([1 << rb] if rb else []) + [16] * (logL // 4)


def dig16(k, logL):
    """Position of frequency k after the DIF stages (digits in the stages' radices)."""
    p, stride = 0, 1 << logL
    for R in radices16(logL):
        stride //= R
        p += (k % R) * stride
        k //= R
    return p


def patterns16(logL):
    L = 1 << logL
    T = L // 16
    rb = logL & 3
    ls0 = logL - (rb if rb else 4)
    pats = [[t + e * T for t in range(T)] for e in range(16)]
    ls = ls0 - 4
    while ls >= 4:
        for r in range(16):
            pats.append([((t >> ls) << (ls + 4)) + (t & ((1 << ls) - 1)) + (r << ls) for t in range(T)])
        ls -= 4
    for r in range(16):
        pats.append([dig16(t, logL) + r for t in range(T)])
    return pats


@pytest.mark.parametrize("es,name", [(8, "kGeoR16_8"), (16, "kGeoR16_16")])
def test_radix16_swizzles_conflict_free(es, name):
    rows = geo_rows(name)
    assert len(rows) == 5
    phase, mask = (16, 15) if es == 8 else (8, 7)
    for logL, prm in zip(range(9, 14), rows):
        L = 1 << logL
        assert sorted(sw(p, prm, es) for p in range(L)) == list(range(L))
        for pat in patterns16(logL):
            for s in range(0, len(pat), phase):
                grp = pat[s:s + phase]
                assert len({sw(p, prm, es) & mask for p in grp}) == len(grp), (logL, prm)


@pytest.mark.parametrize("logL", range(9, 14))
def test_radix16_digit_reversal_groups(logL):
    L = 1 << logL
    assert sorted(dig16(k, logL) for k in range(L)) == list(range(L))
    for t in range(L // 16):
        assert dig16(t, logL) % 16 == 0
        for q in range(16):
            assert dig16(t + q * (L // 16), logL) == dig16(t, logL) + q


def radix16_table(logL):
    """Entries of the radix-16 stage tables as k_twiddles16 writes them: {index: (o, R s)}."""
    rb = logL & 3
    R = (1 << rb) if rb else 16
    s = (1 << logL) // R
    tab, off = {}, 0
    while s > 1:
        for o in range(s):
            tab[off + o] = (o, R * s)
        off += s
        R, s = 16, s // 16
    return tab


@pytest.mark.parametrize("logL", range(9, 14))
def test_radix16_twiddle_offsets(logL):
    L = 1 << logL
    rb = logL & 3
    ls0 = logL - (rb if rb else 4)
    tab = radix16_table(logL)
    assert max(tab) < L
    for t in range(L // 16):  # leading stage: butterflies t + j L/16
        for j in range(16 // ((1 << rb) if rb else 16)):
            assert tab[t + j * (L // 16)] == (t + j * (L // 16), L)
    ls = ls0 - 4
    while ls >= 4:
        off = (1 << ls0) + ((1 << ls0) - (1 << (ls + 4))) // 15  # Fft16::tw_off
        for o in range(1 << ls):
            assert tab[off + o] == (o, 16 << ls)
        ls -= 4


def power_table(logL):
    """Entries of the FP64 power tables as k_twiddles writes them: {index: (o q, R s)}."""
    r0 = logL % 3
    R = (1 << r0) if r0 else 8
    s = (1 << logL) // R
    tab, off = {}, 0
    while True:
        for o in range(s):
            for q in range(1, R):
                tab[off + (q - 1) * s + o] = (o * q, R * s)
        if s == 1:
            break
        off += (R - 1) * s
        R, s = 8, s // 8
    return tab


@pytest.mark.parametrize("logL", range(3, 14))
def test_fp64_power_table_offsets(logL):
    L = 1 << logL
    r0 = logL % 3
    tab = power_table(logL)
    assert max(tab) < L and len(tab) == len(set(tab))
    L8 = L >> 3
    for t in range(L8):  # leading stage as FftC reads it
        if r0 == 0:
            for q in range(1, 8):
                assert tab[(q - 1) * L8 + t] == (t * q, L)
        elif r0 == 2:
            for i in range(2):
                o = t + i * L8
                for q in range(1, 4):
                    assert tab[(q - 1) * (L >> 2) + o] == (o * q, L)
        else:
            for i in range(4):
                o = t + i * L8
                assert tab[o] == (o, L)
    ls = logL - 6 if r0 == 0 else logL - r0 - 3
    while ls >= 3:
        off = ((((1 << r0) - 1) << (logL - r0)) if r0 else 0) + (1 << (logL - r0)) - (8 << ls)  # pow_off
        for o in range(1 << ls):
            for q in range(1, 8):
                assert tab[off + (q - 1) * (1 << ls) + o] == (o * q, 8 << ls)
        ls -= 3


def _dft(v, sgn):
    import numpy as np
    n = len(v)
    k = np.arange(n)
    return np.exp(sgn * 2j * np.pi * np.outer(k, k) / n) @ np.asarray(v)


def _dft16(v, sgn):
    """The 16-point DFT as the kernel's dft16 forms it: DFT-4 over n1 for each n2,
    twiddles w16^(n2 k1), DFT-4 over n2 for each k1, then the 4 x 4 transpose."""
    import numpy as np
    v = np.array(v, dtype=complex)
    for n2 in range(4):
        idx = [n2, n2 + 4, n2 + 8, n2 + 12]
        v[idx] = _dft(v[idx], sgn)
    for n2 in range(4):
        for k1 in range(4):
            v[n2 + 4 * k1] *= np.exp(sgn * 2j * np.pi * n2 * k1 / 16)
    for k1 in range(4):
        v[4 * k1:4 * k1 + 4] = _dft(v[4 * k1:4 * k1 + 4], sgn)
    return np.array([v[4 * (q % 4) + q // 4] for q in range(16)])


def _column_pass16(x, kfull, logL, es, prm):
    """The radix-16 column pass step by step as the kernel runs it (leading stage from
    the thread's points t + e L/16, middle stages in swizzled shared memory, the
    stride-1 stage with the spectrum multiply in registers, the inverse in reverse)."""
    import numpy as np
    L = 1 << logL
    T = L // 16
    rb = logL & 3
    R0 = (1 << rb) if rb else 16
    ls0 = logL - (rb if rb else 4)
    tw = {i: np.exp(-2j * np.pi * o / rs) for i, (o, rs) in radix16_table(logL).items()}
    off = lambda ls: (1 << ls0) + ((1 << ls0) - (1 << (ls + 4))) // 15
    S = lambda p: sw(p, prm, es)
    buf = np.zeros(L, complex)

    def stage0(v, t, inverse):
        sgn = 1 if inverse else -1
        if R0 == 16:
            w = tw[t] ** np.arange(16)
            return _dft16(v * np.conj(w), 1) if inverse else _dft16(v, -1) * w
        J = 16 // R0
        for j in range(J):
            idx = [j + r * J for r in range(R0)]
            w = tw[t + j * T] ** np.arange(R0)
            v[idx] = _dft(v[idx] * np.conj(w), sgn) if inverse else _dft(v[idx], sgn) * w
        return v

    def mid(ls, inverse):
        nb = buf.copy()
        for t in range(T):
            o = t & ((1 << ls) - 1)
            sb = S(((t >> ls) << (ls + 4)) + o)
            ix = [sb ^ S(r << ls) for r in range(16)]
            w = tw[off(ls) + o] ** np.arange(16)
            nb[ix] = _dft16(buf[ix] * np.conj(w), 1) if inverse else _dft16(buf[ix], -1) * w
        return nb

    for t in range(T):
        v = np.zeros(16, complex)
        v[:8] = x[t + np.arange(8) * T]
        buf[[S(t + e * T) for e in range(16)]] = stage0(v, t, False)
    ls = ls0 - 4
    while ls >= 4:
        buf = mid(ls, False)
        ls -= 4
    nb = buf.copy()
    for t in range(T):
        gb = S(dig16(t, logL))
        ix = [gb ^ S(r) for r in range(16)]
        nb[ix] = _dft16(_dft16(buf[ix], -1) * kfull[t + np.arange(16) * T], 1)
    buf = nb
    ls = 4
    while ls <= ls0 - 4:
        buf = mid(ls, True)
        ls += 4
    out = np.zeros(L, complex)
    for t in range(T):
        out[t + np.arange(16) * T] = stage0(buf[[S(t + e * T) for e in range(16)]].copy(), t, True)
    return out


@pytest.mark.parametrize("es,name", [(8, "kGeoR16_8"), (16, "kGeoR16_16")])
@pytest.mark.parametrize("logL", [9, 10, 11, 12])
def test_radix16_column_pass_model(es, name, logL):
    """The column pass's arithmetic (spectrum multiply between a zero-padded forward and a
    cropped inverse transform) in FP64 against numpy's FFT: the decomposition, the
    tables and the swizzled positions together form the circular convolution."""
    import numpy as np
    L = 1 << logL
    rng = np.random.default_rng(logL)
    x = np.zeros(L, complex)
    x[:L // 2] = rng.standard_normal(L // 2) + 1j * rng.standard_normal(L // 2)
    kh = rng.random(L // 2 + 1) + 0.5
    kfull = np.array([kh[k if k <= L // 2 else L - k] for k in range(L)])
    ref = np.fft.ifft(np.fft.fft(x) * kfull) * L
    got = _column_pass16(x, kfull, logL, es, geo_rows(name)[logL - 9])
    assert np.abs(got[:L // 2] - ref[:L // 2]).max() <= 1e-13 * np.abs(ref).max()
