"""Host arithmetic of the CRT residue products against exact integer products, compiled with the host
C++ compiler (no GPU needed): the library's crt.h against 128-bit integers, the wider crt_wide.h
(up to 24 moduli, 84-bit rows) against Python's big integers, and the integer-only conversion of a
128-bit product to FP64 against Python's correctly rounded conversion of the exact rational."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_crt_arithmetic_exact():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "crt_check")
        subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "native", "crt_check.cpp"), "-o", exe],
                       check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout


def _wide_cases(rng):
    """(T, K, pairs) with |F| <= 2^T: random values, all at +2^T (the largest product), +2^T against
    -2^T (the most negative), and a single -1 x 1."""
    cases = []
    for T in (54, 63, 72, 83):
        for K in (1, 2, 64, 1000, 1024, 1025, 16384):
            lim = 1 << T
            for mode in range(4):
                if mode == 0:
                    a = [rng.randrange(-lim, lim + 1) for _ in range(K)]
                    b = [rng.randrange(-lim, lim + 1) for _ in range(K)]
                elif mode == 1:
                    a, b = [lim] * K, [lim] * K
                elif mode == 2:
                    a, b = [lim] * K, [-lim] * K
                else:
                    a, b = [-1] + [0] * (K - 1), [1] + [0] * (K - 1)
                if K == 16384 and mode == 0 and T != 83:
                    continue  # the long random cases once, at the widest rows
                cases.append((T, K, a, b))
    return cases


def test_crt_wide_arithmetic_exact():
    import random
    from fractions import Fraction

    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    rng = random.Random(20240429)
    cases = _wide_cases(rng)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "crt_wide_check")
        subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "native", "crt_wide_check.cpp"), "-o", exe],
                       check=True)
        inp = os.path.join(d, "cases.txt")
        with open(inp, "w") as f:
            for T, K, a, b in cases:
                f.write("%d %d\n" % (T, K))
                m64 = (1 << 64) - 1
                f.write("".join("%d %d %d %d %d %d\n" % (-1 if x < 0 else 1, abs(x) >> 64, abs(x) & m64,
                                                         -1 if y < 0 else 1, abs(y) >> 64, abs(y) & m64)
                                for x, y in zip(a, b)))
        r = subprocess.run([exe, inp], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr
    lines = r.stdout.split("\n")[:len(cases)]
    assert len(lines) == len(cases)
    for (T, K, a, b), line in zip(cases, lines):
        t, k, nmod, got = line.split()
        assert (int(t), int(k)) == (T, K)
        exact = sum(x * y for x, y in zip(a, b))
        want = float(Fraction(exact))
        assert abs(float(got) - want) <= 4 * 2.0 ** -53 * abs(want), (T, K, nmod, got, want)
    # the widest case needs all 24 moduli
    assert any(line.split()[2] == "24" for line in lines)


def test_crt_to_double_correctly_rounded():
    import random
    import struct
    from fractions import Fraction

    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    rng = random.Random(7)
    cases = []
    for _ in range(20000):
        bits = rng.randrange(1, 129)
        x = rng.randrange(1 << (bits - 1), 1 << bits)
        cases.append((rng.choice((-1, 1)), x, rng.randrange(-300, 300)))
    # ties and near-ties around the rounding position, carries into a new binade, tiny and huge values
    for k in (53, 54, 60, 64, 65, 100, 127):
        base = (1 << k) - 1
        cases += [(1, base, 0), (-1, base, -7), (1, (1 << k) + (1 << (k - 53)), 3),
                  (1, (1 << k) + (1 << (k - 53)) + 1, 3), (1, (1 << k) + 3 * (1 << (k - 53)), -40)]
    cases += [(1, 1, 0), (-1, 1, -1000), (1, 3, 1000), (1, (1 << 127) + 1, -200)]
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "crt_convert_check")
        subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "native", "crt_convert_check.cpp"), "-o", exe],
                       check=True)
        inp = os.path.join(d, "cases.txt")
        with open(inp, "w") as f:
            for sg, x, sc in cases:
                f.write("%d %d %d %d\n" % (sg, x >> 64, x & ((1 << 64) - 1), sc))
        r = subprocess.run([exe, inp], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = [struct.unpack("<d", struct.pack("<Q", int(v)))[0] for v in r.stdout.split()]
    assert len(got) == len(cases)
    for (sg, x, sc), g in zip(cases, got):
        want = float(sg * Fraction(x) * Fraction(2) ** sc)
        lo = 2.0 ** -1022
        if abs(want) >= lo or want == 0.0:
            assert g == want, (sg, x, sc, g, want)
        else:   # subnormal results: within one unit of the last place
            assert abs(g - want) <= 2.0 ** -1074, (sg, x, sc, g, want)
