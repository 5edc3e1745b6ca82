"""The identity the kernels use to step coset representatives and tile bases
without depositing every index bit by bit: with an ascending bit list,
deposit(v + G) = ((deposit(v) | ~mask) + deposit(G)) & mask (64-bit words),
as long as v + G still fits the list."""
import random

M64 = (1 << 64) - 1


def deposit(v, bits):
    return sum(((v >> i) & 1) << b for i, b in enumerate(bits))


def walk(x, mask, d):
    return (((x | (~mask & M64)) + d) & M64) & mask


def test_masked_addition_steps_the_deposit():
    rnd = random.Random(7)
    for _ in range(2000):
        n = rnd.randint(1, 63)
        k = rnd.randint(1, n)
        bits = sorted(rnd.sample(range(n), k))
        mask = sum(1 << b for b in bits)
        G = rnd.randint(1, (1 << k) - 1)
        v = rnd.randint(0, (1 << k) - 1 - G) if (1 << k) - 1 - G > 0 else 0
        assert walk(deposit(v, bits), mask, deposit(G, bits)) == deposit(v + G, bits)


def test_walk_visits_a_grid_stride_sequence():
    # a CTA with index c of a grid of size G walks c, c + G, c + 2G, ... as the kernels do
    bits = [3, 5, 6, 9, 13, 20, 31, 40]
    mask = sum(1 << b for b in bits)
    for G in (1, 3, 7, 152):
        for c in range(min(G, 5)):
            x, d = deposit(c, bits), deposit(G, bits)
            for it in range(((1 << len(bits)) - c + G - 1) // G):
                assert x == deposit(c + it * G, bits)
                x = walk(x, mask, d)
