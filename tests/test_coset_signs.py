"""The sign factorisation of the coset kernels, checked on random coset
layouts: staged element e = t + 512 j of the coset with representative rep
is b = rep ^ span(a) ^ l (l = e mod 2^kl, run index a = e >> kl), and
parity(b & z) = parity(rep & z) ^ parity(t & tau) ^ parity(j & w) with
tau = (z mod 2^kl) | (bz mod 2^ash) << kl, w = bz >> ash, ash = 9 - kl, and
bz bit i = parity(basis_i & z).  One Walsh fold over j (level i folds pairs
differing in bit i of j with the sign of bit i of w) gives the signed sum."""
import random


def parity(x):
    return bin(x).count("1") & 1


def test_parity_splits_into_coset_thread_and_element_parts():
    rnd = random.Random(11)
    for _ in range(60):
        n = rnd.randint(15, 40)
        kl = rnd.randint(3, 6)
        m = 13 - kl                                   # 8192 staged = 512 threads x 16 elements
        ash = 9 - kl
        bits = list(range(kl, n))
        rnd.shuffle(bits)
        pivots = sorted(bits[:m])
        basis = []
        for p in pivots:                              # pivot bit p plus random bits above it outside the pivots
            v = 1 << p
            for b in range(p + 1, n):
                if b not in pivots and rnd.random() < 0.3:
                    v |= 1 << b
            basis.append(v)
        free = [b for b in range(kl, n) if b not in pivots]
        rep = sum(1 << b for b in free if rnd.random() < 0.5)
        z = rnd.getrandbits(n)
        bz = sum(parity(basis[i] & z) << i for i in range(m))
        tau = (z & ((1 << kl) - 1)) | ((bz & ((1 << ash) - 1)) << kl)
        w = bz >> ash
        for _ in range(40):
            t, j = rnd.randrange(512), rnd.randrange(16)
            e = t + 512 * j
            a, l = e >> kl, e & ((1 << kl) - 1)
            span = 0
            for i in range(m):
                if (a >> i) & 1:
                    span ^= basis[i]
            b = rep ^ span ^ l
            assert parity(b & z) == parity(rep & z) ^ parity(t & tau) ^ parity(j & w)


def walsh_fold(vals, w):
    vals = list(vals)
    i = 0
    while len(vals) > 1:
        sg = -1.0 if (w >> i) & 1 else 1.0
        vals = [vals[2 * k] + sg * vals[2 * k + 1] for k in range(len(vals) // 2)]
        i += 1
    return vals[0]


def test_walsh_fold_is_the_signed_sum():
    rnd = random.Random(5)
    for N in (2, 4, 8, 16):
        for w in range(N):
            v = [rnd.uniform(-1, 1) for _ in range(N)]
            ref = sum((-1) ** parity(j & w) * v[j] for j in range(N))
            assert abs(walsh_fold(v, w) - ref) < 1e-12
