"""Pins for the oracle's Toeplitz hashing (Sec. III.B standard matrix, Sec. III.D modified matrix).

Every pin here computes the expected value by a route other than the oracle's own formula:
  * the GF(2) polynomial product (Python big integers, shift-and-XOR);
  * the paper's circulant/FFT route (Sec. III.B, Thm. 2; Sec. III.D, the n-point circulant A_c)
    evaluated with numpy's float64 FFT, exact at these sizes;
  * structure the paper states: equal diagonals (Sec. III.B), the identity block of (A, I_m)
    (Sec. III.D), GF(2) linearity, independent blocks (Sec. III.E);
  * brute force over every raw vector for tiny n.
"""
import numpy as np
import pytest

from workloads import pack_bits, random_bits, rng, unpack_bits

STANDARD, MODIFIED = 0, 1


def _seed_len(n, m, form):
    return n + m - 1 if form == STANDARD else n - 1


def _bits(buf, nbits, off=0):
    return unpack_bits(buf, nbits, off).astype(np.int64)


def _poly_int(bits):
    """GF(2)[x] polynomial with coefficient t = bits[t], as a Python int."""
    return int.from_bytes(pack_bits(bits).tobytes(), "little")


def _clmul(a: int, b: int) -> int:
    """Carry-less product of two GF(2) polynomials held in Python ints."""
    out = 0
    while b:
        low = b & -b
        out ^= a << (low.bit_length() - 1)
        b ^= low
    return out


CASES = [(1, 1), (2, 1), (2, 2), (5, 3), (8, 8), (31, 7), (32, 32), (33, 17), (64, 1), (97, 50), (256, 192),
         (300, 299), (1000, 333), (1024, 768), (4096, 2048)]


@pytest.mark.parametrize("n,m", CASES)
def test_standard_equals_polynomial_product(oracle_mod, n, m):
    """k_i is coefficient n-1+i of a(x) r(x) over GF(2): the Toeplitz product is the middle of a
    carry-less polynomial product."""
    g = rng(1000 + n * 7 + m)
    r = _bits(random_bits(n, int(g.integers(1 << 30))), n)
    r[0] = r[-1] = 1  # exercise both edge columns
    raw = pack_bits(r)
    seed = random_bits(n + m - 1, int(g.integers(1 << 30)))
    got = _bits(oracle_mod.toeplitz(raw, n, m, seed, STANDARD), m)
    prod = _clmul(_poly_int(_bits(seed, n + m - 1)), _poly_int(_bits(raw, n)))
    want = np.array([(prod >> (n - 1 + i)) & 1 for i in range(m)])
    assert np.array_equal(got, want)


def _fft_cyclic(a, r):
    """Exact integer cyclic convolution via numpy float64 FFT (small sizes only)."""
    c = np.fft.ifft(np.fft.fft(a.astype(np.float64)) * np.fft.fft(r.astype(np.float64))).real
    ci = np.rint(c)
    assert np.max(np.abs(c - ci)) < 0.25
    return ci.astype(np.int64)


@pytest.mark.parametrize("n,m", [(1, 1), (3, 2), (17, 9), (64, 48), (129, 100), (500, 499), (2048, 1536)])
def test_standard_equals_paper_circulant_route(oracle_mod, n, m):
    """Sec. III.B: embed T in the (n+m-1)-point circulant with first column a, pad r with m-1
    zeros, take F^-1(Fa . Fr'), round, mod 2, keep entries n..n+m-1 (1-based)."""
    g = rng(2000 + n + m)
    L = n + m - 1
    raw = random_bits(n, int(g.integers(1 << 30)))
    seed = random_bits(L, int(g.integers(1 << 30)))
    a = _bits(seed, L)
    r_pad = np.concatenate([_bits(raw, n), np.zeros(m - 1, dtype=np.int64)])
    k_full = _fft_cyclic(a, r_pad) % 2
    want = k_full[n - 1:n - 1 + m]
    got = _bits(oracle_mod.toeplitz(raw, n, m, seed, STANDARD), m)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,m", [(2, 1), (9, 4), (64, 48), (100, 1), (255, 200), (1024, 768), (3000, 1000)])
def test_modified_equals_paper_circulant_route(oracle_mod, n, m):
    """Sec. III.D: n-point circulant A_c with first column a' = (a_1..a_{n-1}, a_n), r' = the first
    n-m raw bits then m zeros, k' = F^-1(Fa' . Fr'), k_i = k'_i + r_{i+1} for n-m <= i <= n-1
    (1-based), mod 2. a_n is arbitrary: both values are tried."""
    g = rng(3000 + n + m)
    raw = random_bits(n, int(g.integers(1 << 30)))
    seed = random_bits(n - 1, int(g.integers(1 << 30)))
    r = _bits(raw, n)
    r_pad = np.concatenate([r[:n - m], np.zeros(m, dtype=np.int64)])
    got = _bits(oracle_mod.toeplitz(raw, n, m, seed, MODIFIED), m)
    for a_n in (0, 1):
        a_prime = np.concatenate([_bits(seed, n - 1), [a_n]])
        k_prime = _fft_cyclic(a_prime, r_pad)
        # 1-based k'_i, i = n-m..n-1  ->  0-based k_prime[i-1]; r_{i+1} -> r[i]
        want = np.array([(k_prime[i - 1] + r[i]) % 2 for i in range(n - m, n)])
        assert np.array_equal(got, want)


@pytest.mark.parametrize("form", [STANDARD, MODIFIED])
@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (8, 5)])
def test_brute_force_all_raw_vectors_linear(oracle_mod, form, n, m):
    """Every raw vector of a tiny block: the map is GF(2)-linear and its columns are the images
    of the unit vectors."""
    seed = random_bits(_seed_len(n, m, form), 77 + n + m + form)
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=np.uint8)
        e[j] = 1
        cols.append(_bits(oracle_mod.toeplitz(pack_bits(e), n, m, seed, form), m))
    cols = np.array(cols).T  # m x n matrix of the hash
    for x in range(1 << n):
        r = np.array([(x >> t) & 1 for t in range(n)], dtype=np.uint8)
        got = _bits(oracle_mod.toeplitz(pack_bits(r), n, m, seed, form), m)
        assert np.array_equal(got, (cols @ r.astype(np.int64)) % 2)


@pytest.mark.parametrize("n,m", [(16, 8), (40, 40), (77, 30)])
def test_standard_columns_are_seed_windows_with_equal_diagonals(oracle_mod, n, m):
    """Sec. III.B: every diagonal of T is constant, and T is fixed by its first row and column,
    which together are the n+m-1 seed bits (T[0][n-1] = a_1 ... T[m-1][0] = a_{n+m-1})."""
    L = n + m - 1
    seed = random_bits(L, 5 * n + m)
    a = _bits(seed, L)
    T = np.zeros((m, n), dtype=np.int64)
    for j in range(n):
        e = np.zeros(n, dtype=np.uint8)
        e[j] = 1
        T[:, j] = _bits(oracle_mod.toeplitz(pack_bits(e), n, m, seed, STANDARD), m)
    assert np.array_equal(T[1:, 1:], T[:-1, :-1])
    assert np.array_equal(T[0, ::-1], a[:n])           # first row read right to left: a_1..a_n
    assert np.array_equal(T[:, 0], a[n - 1:n - 1 + m])  # first column: a_n..a_{n+m-1}


@pytest.mark.parametrize("n,m", [(2, 1), (64, 32), (100, 99), (1000, 750)])
def test_modified_identity_block(oracle_mod, n, m):
    """Sec. III.D: with an all-zero seed only I_m acts, so k = the last m raw bits."""
    raw = random_bits(n, 400 + n)
    seed = np.zeros((n - 1 + 7) // 8, dtype=np.uint8)
    got = _bits(oracle_mod.toeplitz(raw, n, m, seed, MODIFIED), m)
    assert np.array_equal(got, _bits(raw, n)[n - m:])


@pytest.mark.parametrize("n,m", [(10, 4), (128, 96), (999, 500)])
def test_modified_is_standard_on_head_plus_tail(oracle_mod, n, m):
    """(A, I_m) r = A r_head + r_tail, and A is a standard Toeplitz matrix of n-m columns whose
    seed has (n-m)+m-1 = n-1 bits."""
    raw = random_bits(n, 500 + n)
    seed = random_bits(n - 1, 600 + n)
    r = _bits(raw, n)
    head = oracle_mod.toeplitz(pack_bits(r[:n - m]), n - m, m, seed, STANDARD)
    want = (_bits(head, m) + r[n - m:]) % 2
    assert np.array_equal(_bits(oracle_mod.toeplitz(raw, n, m, seed, MODIFIED), m), want)


@pytest.mark.parametrize("form", [STANDARD, MODIFIED])
def test_linearity_random(oracle_mod, form):
    n, m = 777, 300
    seed = random_bits(_seed_len(n, m, form), 9)
    x = random_bits(n, 10)
    y = random_bits(n, 11)
    kx = oracle_mod.toeplitz(x, n, m, seed, form)
    ky = oracle_mod.toeplitz(y, n, m, seed, form)
    kxy = oracle_mod.toeplitz(np.bitwise_xor(x, y), n, m, seed, form)
    assert np.array_equal(np.bitwise_xor(kx, ky), kxy)


@pytest.mark.parametrize("form", [STANDARD, MODIFIED])
def test_blocks_and_selected_bits(oracle_mod, form):
    """Sec. III.E block splitting: the stream helper equals per-block calls at bit offsets, and
    the selected-bit helper equals the matching bits of the full output."""
    n, m, B = 75, 41, 6  # odd sizes: blocks and outputs start mid-byte
    seed = random_bits(_seed_len(n, m, form), 12)
    raw = random_bits(n * B, 13)
    full = oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B)
    for b in range(B):
        one = oracle_mod.toeplitz(raw, n, m, seed, form, raw_off=b * n)
        assert np.array_equal(_bits(one, m), _bits(full, m, b * m))
        idx = np.array([0, 1, m // 2, m - 1], dtype=np.uint64)
        sel = oracle_mod.toeplitz_bits(raw, n, m, seed, form, idx, raw_off=b * n)
        assert np.array_equal(sel, _bits(one, m)[idx.astype(np.int64)])
    if (B * m) % 8:
        assert full[-1] >> ((B * m) % 8) == 0


@pytest.mark.parametrize("form", [STANDARD, MODIFIED])
def test_freivalds_accepts_correct_and_rejects_flipped_bit(oracle_mod, form):
    n, m, B = 200, 120, 9
    seed = random_bits(_seed_len(n, m, form), 14)
    raw = random_bits(n * B, 15)
    out = oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B)
    assert not oracle_mod.freivalds(raw, n, m, seed, form, B, out).any()
    bad = out.copy()
    t = 5 * m + 17
    bad[t // 8] ^= 1 << (t % 8)
    mism = oracle_mod.freivalds(raw, n, m, seed, form, B, bad)
    assert mism[5] != 0 and np.count_nonzero(mism) == 1


def test_rejects_bad_shapes(oracle_mod):
    raw = np.zeros(8, dtype=np.uint8)
    seed = np.zeros(16, dtype=np.uint8)
    with pytest.raises(ValueError):
        oracle_mod.toeplitz(raw, 8, 8, seed, MODIFIED)   # modified needs m < n
    with pytest.raises(ValueError):
        oracle_mod.toeplitz(raw, 8, 0, seed, STANDARD)
