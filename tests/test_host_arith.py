"""Host checks of the integer-valued float arithmetic and the bit tricks the
kernels rely on, over every case the kernels can reach: each kernel states
the claim beside the code, and these tests restate the computation in numpy
with IEEE single-precision rounding and compare it with exact integer
arithmetic.  (The compiled kernels are checked end to end by the GPU parity
tests; these pin the arithmetic arguments themselves.)"""
import numpy as np

f32 = np.float32


def _fma32(a, b, c):
    """fmaf(a, b, c) for float32 arrays: the exact a*b + c (exact in float64
    for the operand sizes used here), rounded once to float32."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _sides():
    """Image sides the library accepts: multiples of 16, 2^a 3^b, up to 768."""
    out = []
    for n in range(16, 769, 16):
        m = n
        while m % 2 == 0:
            m //= 2
        while m % 3 == 0:
            m //= 3
        if m == 1:
            out.append(n)
    return out


def test_fft_small_quotient_is_exact():
    """fdiv_small(x, r) = (int)fmaf(x, r, r / 2) with r = 1/D rounded to float
    gives x / D exactly for 0 <= x <= 16 n and every divisor D of n (the line
    counts n / R and the spans Ns of the Stockham stages; D = n in the CTF
    and FSC passes that split a flat index over at most 16 lines), every
    side n.  The reciprocal is also taken one unit in the last place either
    side, so a reciprocal that is not correctly rounded keeps the result."""
    for n in _sides():
        x = np.arange(0, 16 * n + 1, dtype=np.int64)
        xf = x.astype(f32)
        for D in [k for k in range(1, n + 1) if n % k == 0]:
            r0 = f32(1.0) / f32(D)
            for r in (r0, np.nextafter(r0, f32(0)), np.nextafter(r0, f32(1))):
                rr = np.full_like(xf, r)
                q = _fma32(xf, rr, np.full_like(xf, f32(0.5) * r)).astype(np.int64)  # truncation
                assert np.array_equal(q, x // D), (n, D)


def test_candidate_row_is_exact():
    """candidate_tile: the row of candidate q in a rectangle w tiles wide is
    (int)((q + 1/2) * (1/w)) with both roundings of float32, exact for
    w <= 48 (a 768-pixel side in 16-pixel tiles) and q < 48 w."""
    for w in range(1, 49):
        q = np.arange(0, 48 * w, dtype=np.int64)
        inv = f32(1.0) / f32(w)
        row = ((q.astype(f32) + f32(0.5)) * inv).astype(f32).astype(np.int64)
        assert np.array_equal(row, q // w), w


def test_first_thread_of_a_block_has_margin():
    """Block-aligned forward: a block's first thread is
    floor(((128 - nne) st + 1/2) / N) from a fast division (at most 2 units
    in the last place off).  For every reachable case (nne <= 16 non-empty
    blocks, 0 <= st <= N <= 16 x 256 items) the exact quotient sits at least
    1 / (2 N) from an integer, far more than 4 units in the last place of the
    quotient, so the truncated fast quotient is the exact floor."""
    worst = np.inf
    for N in range(1, 16 * 256 + 1):
        st = np.arange(0, N + 1, dtype=np.int64)
        for nne in (0, 1, 7, 15, 16):
            a = (128 - nne) * st
            v = (a + 0.5) / N
            dist = np.abs(v - np.round(v))
            ulp = np.spacing(v.astype(f32)).astype(np.float64)
            worst = min(worst, float(np.min(dist / ulp)))
            assert np.all(np.floor(v) == a // N)
    assert worst > 4.0, worst


def _transpose_stages(x):
    """The warp's 32 x 32 bit transpose as the kernel computes it: five
    butterfly stages; at stage s lanes j = 16 >> s apart exchange words
    (the xor shuffle), and each keeps its own half of every 2j-bit group
    and takes the partner's other half, shifted by j."""
    x = np.array(x, dtype=np.uint64)
    lane = np.arange(32)
    hi = [0xFFFF0000, 0xFF00FF00, 0xF0F0F0F0, 0xCCCCCCCC, 0xAAAAAAAA]
    for s in range(5):
        j = 16 >> s
        y = x[lane ^ j]
        h = np.uint64(hi[s])
        lo = np.uint64(~hi[s] & 0xFFFFFFFF)
        up = (x & h) | ((y >> np.uint64(j)) & lo)
        dn = (x & lo) | ((y << np.uint64(j)) & h)
        x = np.where((lane & j) != 0, up, dn) & np.uint64(0xFFFFFFFF)
    return x


def test_warp_bit_transpose():
    """After the stages, bit l of lane k is bit k of lane l (lane k < 16
    then holds block k's records of the first 128-record sub-window, lane
    16 + k those of the second, when each lane's word is its two masks)."""
    rng = np.random.default_rng(5)
    cases = [rng.integers(0, 2 ** 32, 32, dtype=np.uint64) for _ in range(200)]
    cases += [np.zeros(32, np.uint64), np.full(32, 0xFFFFFFFF, np.uint64),
              np.array([1 << k for k in range(32)], np.uint64)]
    # two random 16-bit masks per lane, as the forward packs them
    m0 = rng.integers(0, 2 ** 16, 32, dtype=np.uint64)
    m1 = rng.integers(0, 2 ** 16, 32, dtype=np.uint64)
    cases.append(m0 | (m1 << np.uint64(16)))
    for x in cases:
        out = _transpose_stages(x)
        bits_in = (x[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)  # [lane][bit]
        bits_out = (out[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)
        assert np.array_equal(bits_out, bits_in.T)
    # the packed form: lane k < 16 lists the lanes whose first mask has bit k
    out = _transpose_stages(cases[-1])
    for k in range(16):
        assert int(out[k]) == sum(1 << l for l in range(32) if (int(m0[l]) >> k) & 1)
        assert int(out[16 + k]) == sum(1 << l for l in range(32) if (int(m1[l]) >> k) & 1)
