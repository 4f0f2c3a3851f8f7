"""Host-side checks of two invariants the sparse day schedule relies on (the
GPU parity tests check the kernels themselves):

1. Prefix sums of the rates.  The direct method (Appendix A) sums lambda in
   index order and inverts with a running sum over the positive rates whose
   first term is taken as is.  The thread list keeps P_j = (..(w_0 + w_1) +
   ..) + w_j instead and uses P_(T-1) as lambda and P_j as the running sum at
   every positive rate.  That is exact because adding a zero rate (+0 or -0)
   to a positive sum returns the sum, and a sum of zeros plus w returns w.
   Checked here in IEEE double on random rate vectors with zeros of both
   signs, subnormals and wide magnitude ranges.

2. The warp-shared draw buffer.  After a refill with k busy lanes (ranks 0 ..
   k - 1), lane l computes draw c_owner + l // k of the busy unit of rank
   l % k for l < k (32 // k); the unit of rank r reads its draw c + j from
   lane r + j k.  Every busy unit must find each of its 32 // k draws in
   exactly one lane, and no lane index may reach 32.
"""
import numpy as np


def _running_sum_choice(w, target):
    # the inversion as the oracle and fire() write it
    cum, n, last = 0.0, -1, -1
    for j, x in enumerate(w):
        if n < 0 and x > 0.0:
            cum = x if last < 0 else cum + x
            last = j
            if target <= cum:
                n = j
    return last if n < 0 else n


def _prefix(w):
    P, s = [], None
    for j, x in enumerate(w):
        s = x if j == 0 else s + x
        P.append(s)
    return P


def _prefix_choice(w, P, target):
    n, last = -1, -1
    for j, x in enumerate(w):
        if x > 0.0:
            if n < 0:
                last = j
            if n < 0 and target <= P[j]:
                n = j
    return last if n < 0 else n


def _bits(x):
    return np.array([x], dtype=np.float64).view(np.uint64)[0]


def test_prefix_sums_give_lambda_and_the_inversion_bit_for_bit():
    rng = np.random.default_rng(7)
    zeros = [0.0, -0.0]
    for trial in range(20000):
        T = int(rng.integers(1, 9))
        w = []
        for _ in range(T):
            kind = rng.integers(0, 5)
            if kind == 0:
                w.append(zeros[int(rng.integers(0, 2))])
            elif kind == 1:
                w.append(float(rng.uniform(0, 1)) * 2.0 ** -1060)  # subnormal
            else:
                w.append(float(np.exp(rng.uniform(-40, 40))))
        lam = w[0]
        for x in w[1:]:
            lam = lam + x
        P = _prefix(w)
        assert _bits(P[-1]) == _bits(lam)
        if not lam > 0.0:
            continue
        for r2 in (float(rng.random()), 1.0 - 2.0 ** -53, 2.0 ** -53):
            target = lam * r2
            assert _prefix_choice(w, P, target) == _running_sum_choice(w, target)
        # after a transition only rates from j0 on change: recomputing P from
        # j0 equals recomputing it whole
        j0 = int(rng.integers(0, T))
        w2 = list(w)
        for j in range(j0, T):
            if rng.random() < 0.5:
                w2[j] = float(np.exp(rng.uniform(-40, 40)))
        P2 = list(P)
        for j in range(j0, T):
            P2[j] = w2[0] if j == 0 else P2[j - 1] + w2[j]
        assert [_bits(x) for x in P2] == [_bits(x) for x in _prefix(w2)]


def test_draw_buffer_layout_covers_each_busy_unit_once():
    rng = np.random.default_rng(8)
    for trial in range(5000):
        mask = int(rng.integers(1, 2 ** 32))
        busy = [l for l in range(32) if (mask >> l) & 1]
        k = len(busy)
        per = 32 // k
        # refill: lane l holds (owner rank l % k, offset l // k) if l // k < per
        held = {}
        for l in range(32):
            ro, jo = l % k, l // k
            if jo < per:
                assert (ro, jo) not in held
                held[(ro, jo)] = l
        # read: the unit of rank r takes draw c + j from lane r + j k
        for r, lane in enumerate(busy):
            assert bin(mask & ((1 << lane) - 1)).count("1") == r  # its rank
            for j in range(per):
                src = r + j * k
                assert src < 32
                assert held[(r, j)] == src
        assert len(held) == k * per
