"""The float32 identity behind the kernels' integer quantisation of eps
distances on the FMA pipe: for 0 <= p < 2^22, adding 1.5 * 2^23 to p in
float32 (round to nearest, ties to even) lands on the float whose bits are
0x4B400000 + round_half_even(p), the value a float-to-unsigned conversion in
round-to-nearest mode gives.  numpy's float32 addition rounds like the GPU's
__fadd_rn."""
import numpy as np

MAGIC = np.float32(12582912.0)  # 1.5 * 2^23
BIAS = np.uint32(0x4B400000)


def _via_magic(p: np.ndarray) -> np.ndarray:
    return (p.astype(np.float32) + MAGIC).astype(np.float32).view(np.uint32) - BIAS


def test_random_values_match_round_half_even():
    rng = np.random.default_rng(7)
    p = (rng.random(2_000_000) * (2 ** 20 + 8)).astype(np.float32)
    np.testing.assert_array_equal(_via_magic(p), np.rint(p.astype(np.float64)).astype(np.uint32))


def test_ties_go_to_even():
    m = np.arange(0, 2 ** 21, 97, dtype=np.float64)
    p = (m + 0.5).astype(np.float32)  # exact in float32 below 2^22
    expect = np.where(m % 2 == 0, m, m + 1).astype(np.uint32)
    np.testing.assert_array_equal(_via_magic(p), expect)


def test_edges():
    p = np.array([0.0, 0.49999997, 0.5, 1.0, 1.5, 2.5, 2 ** 20, 2 ** 22 - 1], dtype=np.float32)
    np.testing.assert_array_equal(_via_magic(p), np.array([0, 0, 0, 1, 2, 2, 2 ** 20, 2 ** 22 - 1],
                                                          dtype=np.uint32))


def test_round_correction_recovers_the_neighbours_sum():
    """The branch-free kernels add the biased value of min(d2, eps^2) for every
    candidate of a round into a wrapping 32-bit sum; subtracting the bias of
    every slot and the value of eps^2 itself for every candidate beyond eps
    leaves the exact sum over the neighbours (the candidates within eps)."""
    rng = np.random.default_rng(11)
    for e2 in (np.float32(0.0025 * 3), np.float32(0.0025 * 15), np.float32(0.0)):
        scale = np.float32(2 ** 20 / np.sqrt(np.float64(e2))) if e2 > 0 else np.float32(0.0)
        for slots in (4, 1024, 1028):
            d2 = (rng.random(slots) * 3 * max(float(e2), 1e-4)).astype(np.float32)
            d2[rng.random(slots) < 0.05] = e2  # exact boundary hits count as neighbours

            def biased(v):
                p = (np.sqrt(v.astype(np.float32)) * scale).astype(np.float32)
                return (p + MAGIC).astype(np.float32).view(np.uint32)

            capped = np.minimum(d2, e2)
            total = np.uint32(biased(capped).astype(np.uint64).sum() % (1 << 32))
            inside = d2 <= e2
            q_eps = biased(np.array([e2], dtype=np.float32))[0] - BIAS
            got = (int(total) - slots * int(BIAS) - (slots - int(inside.sum())) * int(q_eps)) % (1 << 32)
            expect = int((biased(d2[inside]) - BIAS).astype(np.uint64).sum())
            assert got == expect
