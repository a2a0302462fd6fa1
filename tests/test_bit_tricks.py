"""Word-level identities the kernels rely on, checked on the CPU against their plain
definitions (the kernels themselves are checked against the oracle by the GPU tests).

- Run starts of a row word m: m & ~(m << 1).
- Run ends of m: m & ~(m >> 1); the length of the run starting at x0 is then the
  1-based position of the lowest set bit of (run ends >> x0) (the kernels' __ffs).
- The run starts whose run holds a set bit of c (c within m): c spread towards lower x
  inside each run by doubling -- at the step of shift s, bit i takes bit i + s when m is
  set over [i, i + s] -- then masked with the run starts (the tile pass's face-touch flags).
"""
import random

M = 0xFFFFFFFF


def runs(m):
    out, x = [], 0
    while x < 32:
        if (m >> x) & 1:
            s = x
            while x < 32 and (m >> x) & 1:
                x += 1
            out.append((s, x - s))
        else:
            x += 1
    return out


def run_starts(m):
    return m & ~(m << 1) & M


def touched_starts(m, c):
    c &= m
    f, rr = c, m & (m >> 1)
    for s in (1, 2, 4, 8, 16):
        f |= (f >> s) & rr
        rr &= rr >> s
    return f & run_starts(m)


def test_run_starts():
    rng = random.Random(3)
    for _ in range(20000):
        m = rng.getrandbits(32)
        want = sum(1 << s for s, _ in runs(m))
        assert run_starts(m) == want


def run_ends(m):
    return m & ~(m >> 1) & M


def ffs(v):
    return (v & -v).bit_length()   # 1-based position of the lowest set bit, 0 for none


def test_run_lengths_from_run_ends():
    rng = random.Random(5)
    words = [M, 1, 1 << 31, 0x80000001, 0x55555555, 0xAAAAAAAA, 0x7FFFFFFE, 0xFFFF0000, 0x0000FFFF]
    for t in range(20000):
        m = words[t] if t < len(words) else rng.getrandbits(32) | (rng.getrandbits(32) if t % 2 else 0)
        for s, ln in runs(m):
            assert ffs(run_ends(m) >> s) == ln, (hex(m), s, ln)
            assert s + ffs(run_ends(m) >> s) == s + ln   # one past the last site


def test_touched_run_starts_by_doubling():
    rng = random.Random(1)
    words = [0, M, 1, 1 << 31, 0x80000001, 0x55555555, 0xAAAAAAAA, 0x7FFFFFFE]
    for t in range(100000):
        if t < len(words) ** 2:
            m, c = words[t % len(words)], words[t // len(words)]
        else:
            m = rng.getrandbits(32) | (rng.getrandbits(32) if t % 3 else 0)
            c = rng.getrandbits(32) & rng.getrandbits(32)
        want = 0
        for s, ln in runs(m):
            if ((c & m) >> s) & ((1 << ln) - 1):
                want |= 1 << s
        assert touched_starts(m, c) == want, (hex(m), hex(c))
