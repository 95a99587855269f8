"""CPU model of the register-blocked two-prime NTT passes (the transforms the CUDA
two-prime path runs): the pass plan, the swizzled group addresses, the twiddle-pair
indices and the lazy value bounds, restated in Python and checked against properties
that must hold for any correct plan.

* every pass touches every coefficient exactly once, at the swizzled address of the
  element the butterfly pattern names, inside the polynomial;
* a group's 16-byte accesses start on 4-word boundaries;
* the strided (scalar) accesses of 32 consecutive groups, one warp, hit 32 distinct
  shared-memory banks;
* forward values stay below 4p between stages and below 2p at the end; inverse values
  stay below 2p;
* forward transform, pointwise product, inverse transform and the factor N^{-1} give
  the negacyclic product (schoolbook in full at N = 256 and 512, sampled coefficients at
  N = 1024 and 2048).

This is a model of the kernels' indexing, not the oracle: it shares no code with
either side."""
import random

import pytest

P1, P2 = 998244353, 754974721


def swz(e):
    return e ^ (((e >> 5) & 7) << 2)


def pass_r(logn, s, fwd):
    if logn == 11 and s in (0, 7):
        return 4
    if logn == 10 and ((fwd and s == 0) or (not fwd and s == 6)):
        return 4
    return min(3, logn - s)


def grp_off(logst, r, sb, k):
    c = swz(k << logst)
    m = ((1 << logst) - 1) | ~((1 << (logst + r)) - 1) | 0x1C
    return sb + c if (c & m) == 0 else sb ^ c


def bitrev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


def primitive_root(p):
    m, fs, f = p - 1, [], 2
    while f * f <= m:
        if m % f == 0:
            fs.append(f)
            while m % f == 0:
                m //= f
        f += 1
    if m > 1:
        fs.append(m)
    g = 2
    while any(pow(g, (p - 1) // q, p) == 1 for q in fs):
        g += 1
    return g


def twiddles(p, n, logn):
    """[forward pairs][inverse pairs], each pair (w, floor(w 2^32 / p))."""
    psi = pow(primitive_root(p), (p - 1) // (2 * n), p)
    psi_inv = pow(psi, p - 2, p)
    t = [0] * (4 * n)
    for k in range(n):
        w, wi = pow(psi, bitrev(k, logn), p), pow(psi_inv, bitrev(k, logn), p)
        t[2 * k], t[2 * k + 1] = w, (w << 32) // p
        t[2 * n + 2 * k], t[2 * n + 2 * k + 1] = wi, (wi << 32) // p
    return t


def shoup(x, w, ws, p):
    assert 0 <= x < 2**32
    r = (x * w - ((x * ws) >> 32) * p) % 2**32
    assert r < 2 * p
    return r


def red(a, b):
    return a - b if a >= b else a


def warp_conflicts(addrs_by_group, g):
    """Largest number of distinct words sharing a bank over the warps' scalar accesses."""
    worst = 1
    groups = sorted(addrs_by_group)
    for w0 in range(0, len(groups), 32):
        for k in range(g):
            banks = {}
            for gi in groups[w0:w0 + 32]:
                a = addrs_by_group[gi][k]
                banks.setdefault(a % 32, set()).add(a)
            worst = max(worst, max(len(v) for v in banks.values()))
    return worst


def forward(x, p, t, logn):
    n, s = 1 << logn, 0
    while s < logn:
        r = pass_r(logn, s, True)
        g, logst, lg = 1 << r, logn - s - r, logn - r
        last = s + r == logn
        seen, addrs = set(), {}
        for gidx in range(1 << lg):
            i = gidx >> logst
            x0 = gidx & ((1 << logst) - 1)
            sb = swz((i << (logst + r)) | x0)
            ad = [grp_off(logst, r, sb, k) for k in range(g)]
            e0 = i * (n >> s) + x0
            assert ad == [swz(e0 + (k << logst)) for k in range(g)]
            assert all(0 <= a < n for a in ad)
            if logst == 0 and g >= 4:
                assert all(a % 4 == 0 for a in ad[::4])
            seen.update(ad)
            addrs[gidx] = ad
            v = [x[a] for a in ad]
            for q in range(r):
                half, b = g >> (q + 1), ((1 << s) + i) << q
                w = t[2 * b:2 * b + 2 * (1 << q)]
                for k in range(g):
                    if k & half:
                        continue
                    j = k >> (r - q)
                    vv = shoup(v[k + half], w[2 * j], w[2 * j + 1], p)
                    u = v[k] if (s == 0 and q == 0) else red(v[k], 2 * p)
                    assert u < 2 * p
                    v[k], v[k + half] = u + vv, u - vv + 2 * p
                    assert v[k] < 4 * p and v[k + half] < 4 * p
            if last:
                v = [red(a, 2 * p) for a in v]
            for k in range(g):
                x[ad[k]] = v[k]
        assert len(seen) == n
        if logst > 0 or g < 4:
            assert warp_conflicts(addrs, g) == 1, ("fwd", logn, s, r)
        s += r


def inverse(x, p, t, logn):
    n, s = 1 << logn, 0
    while s < logn:
        r = pass_r(logn, s, False)
        g, lg = 1 << r, logn - r
        seen, addrs = set(), {}
        for gidx in range(1 << lg):
            i = gidx >> s
            x0 = gidx & ((1 << s) - 1)
            sb = swz((i << (s + r)) | x0)
            ad = [grp_off(s, r, sb, k) for k in range(g)]
            e0 = (i << (s + r)) + x0
            assert ad == [swz(e0 + (k << s)) for k in range(g)]
            assert all(0 <= a < n for a in ad)
            seen.update(ad)
            addrs[gidx] = ad
            v = [x[a] for a in ad]
            for q in range(r):
                dist, nb = 1 << q, 1 << (r - 1 - q)
                b = (n >> (s + q + 1)) + (i << (r - 1 - q))
                assert b % nb == 0
                w = t[2 * n + 2 * b:2 * n + 2 * b + 2 * nb]
                for k in range(g):
                    if k & dist:
                        continue
                    j = k >> (q + 1)
                    u, vv = v[k], v[k + dist]
                    assert u < 2 * p and vv < 2 * p
                    v[k] = red(u + vv, 2 * p)
                    v[k + dist] = shoup(u - vv + 2 * p, w[2 * j], w[2 * j + 1], p)
            for k in range(g):
                x[ad[k]] = v[k]
        assert len(seen) == n
        if s > 0 or g < 4:
            assert warp_conflicts(addrs, g) == 1, ("inv", logn, s, r)
        s += r


def negacyclic_coef(a, b, e, p):
    n = len(a)
    return sum(a[i] * b[(e - i) % n] * (1 if i <= e else -1) for i in range(n)) % p


@pytest.mark.parametrize("logn", [8, 9, 10, 11])
@pytest.mark.parametrize("p", [P1, P2])
def test_pass_plan_product(logn, p):
    n = 1 << logn
    rng = random.Random(logn * 7 + p % 13)
    t = twiddles(p, n, logn)
    a = [rng.randrange(p) for _ in range(n)]
    b = [rng.randrange(p) for _ in range(n)]
    sa, sb_ = [0] * n, [0] * n
    for e in range(n):
        sa[swz(e)], sb_[swz(e)] = a[e], b[e]
    forward(sa, p, t, logn)
    forward(sb_, p, t, logn)
    assert all(v < 2 * p for v in sa + sb_)
    c = [(sa[k] * sb_[k]) % p for k in range(n)]
    inverse(c, p, t, logn)
    ninv = pow(n, p - 2, p)
    got = [(c[swz(e)] * ninv) % p for e in range(n)]
    coefs = range(n) if logn <= 9 else rng.sample(range(n), 6) + [0, n - 1]
    for e in coefs:
        assert got[e] == negacyclic_coef(a, b, e, p), (logn, p, e)
