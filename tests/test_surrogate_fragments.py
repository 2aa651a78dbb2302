"""The learned tail's tensor-core operands, checked on the host.

steps_cyl_surrogate_lanes returns the per-lane records that the surrogate
kernels stage in shared memory and the output shift they add. This test runs
those records through an emulation of the PTX mma.sync fragment layouts
(m16n8k8 and m16n8k16 with f16 operands: lane 4g + t holds A rows g and g + 8 at
columns 2t, 2t + 1 (and 2t + 8, 2t + 9), B column g at rows 2t, 2t + 1 (and
2t + 8, 2t + 9), and C/D rows g and g + 8 at columns 2t, 2t + 1), in the order the
kernel's network takes them:
- the inputs staged so that m-tile mt holds the pairs of lanes 4g + 2mt (row g)
  and 4g + 2mt + 1 (row g + 8), with (u0, u1), (u2, 1) and zeros as columns;
- ReLU and FP16 packing of each accumulator into the next layer's A operand;
- the two tiles' output products added into one accumulator, a lane reading its
  own pair's outputs from row g + 8 (t & 1).
The result must equal the network of the parameter vector evaluated directly,
with the same roundings: FP16 weights, inputs and activations, b1 as an FP16
weight, b2 in FP32, and b3 through the shift mu + sc b3. A transposed fragment,
a swapped tile or a wrong column in any layer moves the outputs by O(1), which
a planted swap below confirms."""
import numpy as np
import pytest

from paper_2602_20787_gb300 import ics

H = 32


def f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def halves(word):
    """An f16x2 word as (low, high) values."""
    w = np.array([word], dtype=np.uint32)
    return tuple(w.view(np.float16).astype(np.float64))


def mma(a, b, c, k):
    """D = A B + C of one warp, from per-lane fragments: a[L] (f16 pairs), b[L]
    (f16 pairs), c[L] (4 values); returns d[L] (4 values)."""
    A, B, C = np.zeros((16, k)), np.zeros((k, 8)), np.zeros((16, 8))
    for L in range(32):
        g, t = L >> 2, L & 3
        A[g, 2 * t:2 * t + 2], A[g + 8, 2 * t:2 * t + 2] = a[L][0], a[L][1]
        B[2 * t:2 * t + 2, g] = b[L][0]
        if k == 16:
            A[g, 2 * t + 8:2 * t + 10], A[g + 8, 2 * t + 8:2 * t + 10] = a[L][2], a[L][3]
            B[2 * t + 8:2 * t + 10, g] = b[L][1]
        C[g, 2 * t:2 * t + 2], C[g + 8, 2 * t:2 * t + 2] = c[L][0:2], c[L][2:4]
    D = A @ B + C
    return [[D[L >> 2, 2 * (L & 3)], D[L >> 2, 2 * (L & 3) + 1], D[(L >> 2) + 8, 2 * (L & 3)],
             D[(L >> 2) + 8, 2 * (L & 3) + 1]] for L in range(32)]


def relu_pack(lo, hi):
    return (f16(max(lo, 0.0)), f16(max(hi, 0.0)))


def network_from_lanes(lanes, u):
    """The network outputs (without b3) of one warp for one value of j: u[L] are
    lane L's inputs; returns y[L] (2 values) for lane L's own pair."""
    w = lambda L, i: halves(lanes[L, i])
    zero = [[0.0] * 4] * 32
    # input staging: slot 0 (u0, u1), slot 1 (u2, 1), slots 2 and 3 zero; lane
    # (g, t) reads the words of lanes 4g .. 4g + 3 in slot t
    slot = [[(f16(u[L][0]), f16(u[L][1])) for L in range(32)], [(f16(u[L][2]), 1.0) for L in range(32)],
            [(0.0, 0.0)] * 32, [(0.0, 0.0)] * 32]
    inp = [[slot[L & 3][4 * (L >> 2) + q] for q in range(4)] for L in range(32)]
    a2 = []
    for mt in range(2):
        d1 = [mma([[inp[L][2 * mt], inp[L][2 * mt + 1]] for L in range(32)], [[w(L, nb)] for L in range(32)], zero, 8)
              for nb in range(4)]
        a2.append([[[relu_pack(d1[2 * kb][L][0], d1[2 * kb][L][1]), relu_pack(d1[2 * kb][L][2], d1[2 * kb][L][3]),
                     relu_pack(d1[2 * kb + 1][L][0], d1[2 * kb + 1][L][1]),
                     relu_pack(d1[2 * kb + 1][L][2], d1[2 * kb + 1][L][3])] for kb in range(2)] for L in range(32)])
    a3 = [[[[None] * 4 for _ in range(2)] for _ in range(32)] for _ in range(2)]
    for nb in range(4):
        c2 = [[float(np.uint32(lanes[L, 28 + 4 * nb + q]).view(np.float32)) for q in range(4)] for L in range(32)]
        for mt in range(2):
            d = mma([a2[mt][L][0] for L in range(32)], [[w(L, 4 + 4 * nb), w(L, 5 + 4 * nb)] for L in range(32)],
                    c2, 16)
            d = mma([a2[mt][L][1] for L in range(32)], [[w(L, 6 + 4 * nb), w(L, 7 + 4 * nb)] for L in range(32)],
                    d, 16)
            for L in range(32):
                a3[mt][L][nb >> 1][2 * (nb & 1)] = relu_pack(d[L][0], d[L][1])
                a3[mt][L][nb >> 1][2 * (nb & 1) + 1] = relu_pack(d[L][2], d[L][3])
    d = zero
    for mt, base in ((0, 20), (1, 24)):
        for kb in range(2):
            d = mma([a3[mt][L][kb] for L in range(32)],
                    [[w(L, base + 2 * kb), w(L, base + 2 * kb + 1)] for L in range(32)], d, 16)
    return np.array([(d[L][2], d[L][3]) if (L & 1) else (d[L][0], d[L][1]) for L in range(32)])


def network_direct(P, u):
    """The same network from the parameter vector: W1[32][3], b1, W2[32][32], b2,
    W3[2][32], b3 (not added), with the kernel's roundings."""
    P = P.astype(np.float64)
    W1, b1 = P[0:96].reshape(H, 3), P[96:128]
    W2, b2 = P[128:1152].reshape(H, H), P[1152:1184]
    W3 = P[1184:1248].reshape(2, H)
    h1 = f16(np.maximum(f16(W1) @ f16(u) + f16(b1), 0.0))
    h2 = f16(np.maximum(f16(W2) @ h1 + b2, 0.0))
    return f16(W3) @ h2


@pytest.fixture(scope="module")
def sc():
    from paper_2602_20787_gb300 import build, steps_cyl
    build.build()
    return steps_cyl


@pytest.mark.parametrize("seed", [3, 17])
def test_kernel_operands_give_the_network(sc, seed):
    P = ics.random_surrogate_params(seed, 8.0, mu=(0.02, -0.01), sc=(0.05, 0.03))
    lanes, shift = sc.steps_cyl_surrogate_lanes(P)
    assert lanes.shape == (32, sc.STEPS_SURR_LANE_WORDS)
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, (32, 3))
    y = network_from_lanes(lanes, u)
    ref = np.array([network_direct(P, u[L]) for L in range(32)])
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(y - ref).max()
    # the output bias enters through the shift: E (sc (y + b3) + mu) = E (sc y + shift)
    b3, mu, scale = P[1248:1250].astype(np.float64), P[1250:1252].astype(np.float64), P[1252:1254].astype(np.float64)
    np.testing.assert_array_equal(shift, (mu + scale * b3).astype(np.float32))
    # a planted mistake: the two m-tiles' output operands swapped between lanes
    bad = lanes.copy()
    bad[:, 20:24], bad[:, 24:28] = lanes[:, 24:28], lanes[:, 20:24]
    assert np.abs(network_from_lanes(bad, u) - ref).max() > 1e-3 * np.abs(ref).max()


def test_refuses_null_and_wrong_size(sc):
    with pytest.raises(sc.StepsError):
        sc.steps_cyl_surrogate_lanes(np.zeros(10, dtype=np.float32))
    L = sc.load()
    assert L.steps_cyl_surrogate_lanes(None, None, None) == sc.STEPS_EINVAL
