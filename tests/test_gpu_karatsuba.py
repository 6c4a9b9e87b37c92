"""GPU parity of the block-Karatsuba route (QRNG_ALGO_GEMM_KARATSUBA) against the oracle, for
every split depth and block side the route accepts. The route reorganises the GF(2) product of
Sec. III.B / III.D (2x2 Toeplitz blocks in three products, parities XOR-combined), so its output
must equal the definition bit for bit. Shapes: ragged m and n (zero-padded rows and columns),
several row blocks (the seed window moves by span - h per block), several block-column tiles
(B > 224) and passes split by a small workspace budget."""
import numpy as np
import pytest

import workloads as W
from gpu_util import extract, spot_check

pytestmark = pytest.mark.gpu

STD, MOD = 0, 1
KARA = 8  # QRNG_ALGO_GEMM_KARATSUBA


def _case(n, m, form, B, s):
    raw = W.random_bits(n * B, 4000 + s)
    seed = W.random_bits(n + m - 1 if form == STD else n - 1, 5000 + s)
    return raw, seed


@pytest.fixture
def kara(qlib, gpu):
    yield lambda levels, h, ws=0: qlib.qrng_set_karatsuba(gpu, levels, h, ws)
    qlib.qrng_set_karatsuba(gpu, 0, 0, 0)


SPLITS = [(1, 256), (2, 256), (3, 256), (4, 256), (1, 512), (2, 512), (3, 512), (4, 512), (1, 1024), (2, 1024),
          (3, 1024), (1, 2048), (2, 2048), (1, 4096), (1, 8192)]
SHAPES = [(5000, 3100, STD, 3), (5000, 3100, MOD, 230), (9000, 5000, STD, 2), (4500, 1700, MOD, 5),
          (3000, 2900, STD, 4), (2048, 1024, STD, 1), (700, 300, MOD, 3), (1, 1, STD, 2), (33, 17, MOD, 2)]


@pytest.mark.parametrize("levels,h", SPLITS)
@pytest.mark.parametrize("n,m,form,B", SHAPES)
def test_forced_splits_bit_exact(qlib, gpu, oracle_mod, kara, levels, h, n, m, form, B):
    kara(levels, h)
    raw, seed = _case(n, m, form, B, n + 7 * m + B + levels)
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B)
    got = extract(qlib, gpu, raw, n, m, seed, form, KARA, B)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("levels,h", [(2, 1024), (3, 512), (2, 512), (3, 256), (2, 256), (4, 256)])
def test_laser_shape_several_blocks(qlib, gpu, oracle_mod, kara, levels, h):
    """The laser-stream block shape (n = 2^16, m = 36,473): nine row blocks of 1024 at two levels,
    sixteen K blocks; the sub-product sums reach 2^14 per accumulator."""
    n, m, B = 1 << 16, 36473, 3
    kara(levels, h)
    raw, seed = _case(n, m, STD, B, 77 + levels)
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, STD, B)
    assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, STD, KARA, B), want)


@pytest.mark.parametrize("levels,h", [(2, 512), (2, 256), (4, 256)])
def test_chunked_passes(qlib, gpu, oracle_mod, kara, levels, h):
    """A workspace budget of one 224-block pass: 700 blocks run in four passes whose outputs land
    at their blocks' places."""
    n, m, B = 4096, 3000, 700
    kara(levels, h, 1)  # below one block's need: the pass holds the minimum of 224 blocks
    raw, seed = _case(n, m, MOD, B, 11)
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, MOD, B)
    assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, MOD, KARA, B), want)


def test_many_blocks_match_direct(qlib, gpu, oracle_mod, kara):
    """Full occupancy: 76 clusters with several tiles each, repeated; equal to the direct kernel,
    whose output is checked against the oracle on every block."""
    n, m, B = 1 << 14, 12000, 224 * 9 + 5
    raw, seed = _case(n, m, STD, B, 13)
    ref = extract(qlib, gpu, raw, n, m, seed, STD, qlib.QRNG_ALGO_DIRECT, B)
    assert not oracle_mod.freivalds(raw, n, m, seed, STD, B, ref).any()
    for levels, h in ((2, 1024), (3, 512), (3, 256), (4, 256), (0, 0)):
        kara(levels, h)
        for _ in range(2):
            assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, STD, KARA, B), ref)


def test_all_ones_derived_operands(qlib, gpu, oracle_mod, kara):
    """All-ones raw and seed: every derived operand of a B or C product and every XOR of two raw
    blocks is zero inside the matrix, so the output is the parity of n on every row."""
    n, m, B = 1 << 16, 20000, 4
    raw = np.full(n * B // 8, 0xFF, dtype=np.uint8)
    seed = W.pack_bits(np.ones(n + m - 1, dtype=np.uint8))
    for levels, h in ((1, 512), (2, 1024), (3, 2048), (3, 256), (4, 256)):
        kara(levels, h)
        got = extract(qlib, gpu, raw, n, m, seed, STD, KARA, B)
        assert np.array_equal(np.unpackbits(got, bitorder="little")[:m * B], np.zeros(m * B, np.uint8) + (n & 1))


def test_long_blocks_spot_checked(qlib, gpu, oracle_mod, kara):
    """n_t = 2^22 - 96 (the tensor-core limit, ragged), one row block."""
    n, m, B = (1 << 22) - 96, 1000, 2
    raw, seed = _case(n, m, STD, B, 17)
    for levels, h in ((0, 0), (2, 512), (2, 256), (4, 256)):
        kara(levels, h)
        got = extract(qlib, gpu, raw, n, m, seed, STD, KARA, B)
        spot_check(oracle_mod, raw, n, m, seed, STD, got, blocks=[0, B - 1], per_block=96)


@pytest.mark.parametrize("levels,h", [(-1, 0), (5, 0), (1, 128), (1, 3000), (2, 16384)])
def test_bad_settings_rejected(qlib, gpu, levels, h):
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_set_karatsuba(gpu, levels, h, 0)
    assert e.value.status == qlib.QRNG_EINVAL


def test_plan_query(qlib, gpu, kara):
    """qrng_karatsuba_plan reports the shape the route runs: 3^L sub-products whose sides are the
    h-blocks of every span-th position of the padded matrix (an even number of row blocks when
    h = 256), and the forced settings when they are set."""
    n, m, B = 1 << 16, 36473, 8192
    p = qlib.qrng_karatsuba_plan(gpu, n, m, STD, B)
    L, h = p["levels"], p["h"]
    span = h << L
    assert 1 <= L <= 4 and p["groups"] == 3 ** L
    rblocks = -(-m // span)
    if h == 256:
        rblocks += rblocks & 1
    assert p["mq"] == rblocks * h and p["kq"] == -(-n // span) * h
    assert p["blocks_per_pass"] == B and p["model_s"] > 0
    kara(2, 1024)
    p = qlib.qrng_karatsuba_plan(gpu, n, m, MOD, B)
    assert (p["levels"], p["h"], p["groups"], p["mq"], p["kq"]) == (2, 1024, 9, 9 * 1024, 8 * 1024)
    with pytest.raises(qlib.QrngError) as e:
        qlib.qrng_karatsuba_plan(gpu, 64, 65, STD, 1)
    assert e.value.status == qlib.QRNG_EINVAL


@pytest.mark.parametrize("levels,h", [(0, 0), (1, 256), (2, 512), (3, 256), (4, 256)])
@pytest.mark.parametrize("n,m,form,B", [
    (4096, 100, STD, 32), (5000, 3100, STD, 8), (1 << 16, 36473, STD, 32), (4500, 1700, MOD, 16),
    (3000, 99, STD, 31),  # 3069 output bits: the last byte has three pad bits
])
def test_combination_writes_the_packed_stream(qlib, gpu, oracle_mod, kara, levels, h, n, m, form, B):
    """Shapes whose packed output is 4-byte aligned and a whole number of words long with m not a
    multiple of 32: the combination pass writes the bit stream in place, blocks meeting inside
    words (AND/OR on the shared words), the pad bits of the last byte zeroed, nothing written past
    the stream."""
    kara(levels, h)
    raw, seed = _case(n, m, form, B, 3 * m + B + levels)
    assert ((B * m + 7) // 8) % 4 == 0
    got = extract(qlib, gpu, raw, n, m, seed, form, KARA, B)
    if n * m <= 1 << 24:
        assert np.array_equal(got, oracle_mod.toeplitz_blocks(raw, n, m, seed, form, B))
    else:  # the laser shape: every block by Freivalds, block edges and pad bits bit by bit
        assert not oracle_mod.freivalds(raw, n, m, seed, form, B, got).any()
        spot_check(oracle_mod, raw, n, m, seed, form, got, blocks=range(B), per_block=16)
        tail = (B * m) % 8
        if tail:
            assert got[-1] >> tail == 0


def test_packed_stream_over_passes(qlib, gpu, oracle_mod, kara):
    """The in-place combination over several passes (blocks numbered across passes)."""
    n, m, B = 4096, 1000, 704  # 88,000 bytes; a pass holds 224 blocks
    kara(2, 256, 1)
    raw, seed = _case(n, m, STD, B, 19)
    want = oracle_mod.toeplitz_blocks(raw, n, m, seed, STD, B)
    assert np.array_equal(extract(qlib, gpu, raw, n, m, seed, STD, KARA, B), want)
