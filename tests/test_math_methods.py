"""The numerical methods behind the descriptors' per-neighbour factors, checked
on the CPU (no GPU): each method is re-evaluated here step by step in float32
(numpy, round to nearest; an FMA as one rounding of the exact product-sum) and
compared with FP64.  This pins the methods' design: the reduction, the series
coefficients (ln 2)^k / k!, the table of cos/sin(pi k/64) and the double-float
bookkeeping, including that the high half of each double-float result is by
itself accurate (a force-pass derivative uses it alone).  The device code is
checked against closed forms on the GPU (test_gpu_accuracy.py)."""
import math

import numpy as np

F = np.float32
U = 2.0 ** -24
C = [1.3215486790144305e-06, 1.5252733804059838e-05, 1.5403530393381606e-04, 1.3333558146428441e-03,
     9.6181291076284772e-03, 5.5504108664821576e-02, 2.4022650695910071e-01, 6.9314718055994531e-01, 1.0]


def fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def exp2_acc(x):
    """2^x: x = n + f, |f| <= 1/2, Taylor series of e^(f ln 2) to degree 8, scaled by 2^n."""
    x = F(min(max(x, -125.0), 127.0))
    n = F(np.rint(x))
    f = F(x - n)
    p = F(C[0])
    for c in C[1:]:
        p = fma(p, f, F(c))
    return F(p * F(2.0 ** int(n)))


def exp2_dd(ah, al):
    ah = F(min(max(ah, -125.0), 127.0))
    n = F(np.rint(ah))
    f, fl = two_sum(F(ah - n), F(al))
    q = F(C[0])
    for c in C[1:7]:
        q = fma(q, f, F(c))
    ln2h, ln2l = F(6.93147182464599609375e-01), F(-1.9046542999577e-09)
    th = F(f * ln2h)
    tl = F(fma(f, ln2h, -th) + fma(f, ln2l, fma(fl, ln2h, F(F(f * f) * q))))
    sh = F(F(1.0) + th)
    sl = F(F(F(F(1.0) - sh) + th) + tl)
    rh = F(sh + sl)
    rl = F(sl - F(rh - sh))
    sc = F(2.0 ** int(n))
    return F(rh * sc), F(rl * sc)


TAB = []
for k in range(33):
    c, s = math.cos(math.pi * k / 64), math.sin(math.pi * k / 64)
    TAB.append((F(c), F(c - float(F(c))), F(s), F(s - float(F(s)))))


def cospi_dd(xh, xl):
    k = int(min(max(np.rint(F(xh * F(64.0))), 0), 32))
    t = TAB[k]
    dd = F(F(xh - F(F(k) * F(0.015625))) + F(xl))
    a = fma(dd, F(-8.742278e-08), F(dd * F(3.14159274101257324)))
    a2 = F(a * a)
    omc = F(a2 * fma(a2, F(-4.16666679e-02), F(0.5)))
    sna = F(a * fma(a2, F(-1.66666672e-01), F(1.0)))
    D = F(fma(t[0], omc, F(t[2] * sna)) - t[1])
    ch, cl = two_sum(t[0], -D)
    sn = F(t[2] + fma(t[0], sna, -F(t[2] * omc)))
    return ch, cl, sn


def test_exp2_acc_unbiased_and_within_an_ulp():
    xs = np.random.default_rng(1).uniform(-20.0, 0.0, 4000)
    e = np.array([(float(exp2_acc(F(x))) - 2.0 ** float(F(x))) / 2.0 ** float(F(x)) for x in xs]) / U
    assert abs(e.mean()) < 0.05 and np.sqrt(np.mean(e ** 2)) < 0.6 and np.abs(e).max() < 1.2


def test_exp2_dd_pair_and_high_half():
    rng = np.random.default_rng(2)
    xs = rng.uniform(-20.0, 0.0, 3000)
    pair, high = [], []
    for x in xs:
        ah = F(x)
        al = F(rng.uniform(-1, 1) * 1e-7 * abs(float(ah)))
        want = 2.0 ** (float(ah) + float(al))
        h, l = exp2_dd(ah, al)
        pair.append((float(h) + float(l) - want) / want)
        high.append((float(h) - want) / want)
    pair, high = np.array(pair) / U, np.array(high) / U
    assert np.abs(pair).max() < 0.2          # ~2^-27 relative
    assert np.abs(high).max() < 1.0          # the high half alone within an ulp


def test_cospi_dd_absolute_and_sin():
    rc = 5.5
    inv = 1.0 / (2.0 * rc)
    ih = F(inv)
    il = F(inv - float(ih))
    worst_c, worst_s = 0.0, 0.0
    for r in np.linspace(0.3, rc - 1e-3, 3000):
        rh = F(r)
        xh = F(rh * ih)
        xl = F(fma(rh, ih, -xh) + fma(rh, il, F(0.0)))
        ch, cl, sn = cospi_dd(xh, xl)
        x = float(rh) / (2.0 * rc)
        worst_c = max(worst_c, abs(float(ch) + float(cl) - math.cos(math.pi * x)))
        worst_s = max(worst_s, abs(float(sn) - math.sin(math.pi * x)) / math.sin(math.pi * x))
    assert worst_c < 0.1 * U      # cos(pi x) as hi + lo to ~2^-28 absolute
    assert worst_s < 2.0 * U      # sin(pi x) to ~1 ulp


def test_cospi_dd_table_endpoints():
    for k in (0, 32):
        x = k / 64.0
        ch, cl, _ = cospi_dd(F(x), F(0.0))
        assert abs(float(ch) + float(cl) - math.cos(math.pi * x)) < 1e-15
