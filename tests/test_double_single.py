"""The double-single arithmetic of the OC bisection passes, emulated on the
CPU with float32 arrays in the kernel's order of operations: q, lo, hi and
the candidate factor t = 1/sqrt(lambda) as pairs of floats, the product by
the FMA error term, the clamp by comparing pairs, the sum by two-sum with
the rounding error carried in the low word.  Checked against the FP64 clamp
sum of the OC update (Section 2.3): the design volume at a candidate must
come out within 1e-12 relative, the accuracy the bisection's decisions
rely on.  (A float32 FMA is emulated exactly where the kernel needs it to
be exact: the error of a float32 product is a float32 and the float64
product is exact.)"""
import numpy as np

f32 = np.float32


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _ds(v):
    h = v.astype(f32)
    return h, (v - h.astype(np.float64)).astype(f32)


def _ds_mul(ah, al, bh, bl):
    p = (ah * bh).astype(f32)
    e = _fma(ah, bh, -p)                   # exact error of the leading product
    e = _fma(ah, bl, e)
    e = _fma(al, bh, e)
    s = (p + e).astype(f32)
    return s, (e - (s - p)).astype(f32)


def _ds_lt(ah, al, bh, bl):
    return (ah < bh) | ((ah == bh) & (al < bl))


def _ds_acc(ah, al, vh, vl):
    s = (ah + vh).astype(f32)
    bb = (s - ah).astype(f32)
    err = ((ah - (s - bb)) + (vh - bb)).astype(f32)
    lo = ((al + err) + vl).astype(f32)
    h2 = (s + lo).astype(f32)
    return h2, (lo - (h2 - s)).astype(f32)


def _volume_ds(q, lo, hi, t, threads=64):
    """Per 'thread' a double-single running sum over its grid-stride
    elements, then FP64 across threads (the kernel's layout)."""
    qh, ql = _ds(q)
    lh, ll = _ds(lo)
    hh, hl = _ds(hi)
    th, tl = _ds(np.array([t]))
    n = len(q)
    steps = -(-n // threads)
    pad = steps * threads - n
    arrs = [np.concatenate([a, np.zeros(pad, a.dtype)]).reshape(steps, threads)
            for a in (qh, ql, lh, ll, hh, hl)]
    ah = np.zeros(threads, f32)
    al = np.zeros(threads, f32)
    for k in range(steps):
        a_qh, a_ql, a_lh, a_ll, a_hh, a_hl = (a[k] for a in arrs)
        vh, vl = _ds_mul(a_qh, a_ql, np.full(threads, th[0]), np.full(threads, tl[0]))
        below = _ds_lt(vh, vl, a_lh, a_ll)
        above = _ds_lt(a_hh, a_hl, vh, vl)
        ch = np.where(below, a_lh, np.where(above, a_hh, vh))
        cl = np.where(below, a_ll, np.where(above, a_hl, vl))
        ah, al = _ds_acc(ah, al, ch, cl)
    return float(np.sum(ah.astype(np.float64) + al.astype(np.float64)))


def test_double_single_volume_matches_fp64_clamp_sum():
    rng = np.random.Generator(np.random.PCG64(7))
    n = 6000
    x = rng.uniform(1e-3, 1.0, n)
    dc = -rng.lognormal(0.0, 3.0, n)
    q = x * np.sqrt(-dc)
    lo = np.maximum(0.0, x - 0.2)
    hi = np.minimum(1.0, x + 0.2)
    q[:50] = 0.0                          # passive elements: q = lo = hi = 0
    lo[:50] = hi[:50] = 0.0
    for lam in (5e8, 1e3, 3.7, 0.1234567, 1e-4, 1e-9):
        t = 1.0 / np.sqrt(lam)
        ref = np.clip(q * t, lo, hi).sum()
        got = _volume_ds(q, lo, hi, t)
        assert abs(got - ref) <= 1e-12 * ref, (lam, got, ref)


def test_double_single_clamp_picks_the_fp64_branch():
    """Away from ties (relative gaps above 1e-12), the pair comparison takes
    the same branch of the clamp as FP64 does."""
    rng = np.random.Generator(np.random.PCG64(8))
    q = rng.uniform(0.0, 3.0, 20000)
    lo = rng.uniform(0.0, 0.5, 20000)
    hi = lo + rng.uniform(0.0, 0.5, 20000)
    t = 0.7316
    prod = q * t
    th, tl = _ds(np.array([t]))
    qh, ql = _ds(q)
    vh, vl = _ds_mul(qh, ql, np.full(len(q), th[0]), np.full(len(q), tl[0]))
    lh, ll = _ds(lo)
    hh, hl = _ds(hi)
    below = _ds_lt(vh, vl, lh, ll)
    above = _ds_lt(hh, hl, vh, vl)
    far = (np.abs(prod - lo) > 1e-12 * np.maximum(prod, 1e-300)) & \
          (np.abs(prod - hi) > 1e-12 * np.maximum(prod, 1e-300))
    assert np.array_equal(below[far], (prod < lo)[far])
    assert np.array_equal(above[far], (prod > hi)[far])
