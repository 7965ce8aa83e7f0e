"""The packing kernels' inner step (csrc/pack_bits.cuh), compiled for the
host with g++ and checked against the plain byte-wise rule: a byte is a
base when it is A, C, G or T in either case, its 2-bit code is
(byte >> 1) & 3 (hi plane = code bit 1, lo plane = code bit 0), and any
other byte sets the N plane with both code bits cleared.  Every byte value
at every one of the 32 positions (the rest random bases), then random
mixes of bases, N, IUPAC letters and arbitrary bytes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_27291_b300", "csrc")

PROGRAM = r"""
#include "pack_bits.cuh"
#include <cstdio>
#include <cstring>
#include <random>

static void rule(const unsigned char *s, uint32_t &hi, uint32_t &lo, uint32_t &nn) {
    hi = lo = nn = 0;
    for (int b = 0; b < 32; b++) {
        const unsigned u = s[b] & 0xDFu;
        const bool base = u == 'A' || u == 'C' || u == 'G' || u == 'T';
        const unsigned code = base ? (s[b] >> 1) & 3u : 0u;
        hi |= (code >> 1) << b;
        lo |= (code & 1u) << b;
        nn |= (base ? 0u : 1u) << b;
    }
}

int main() {
    std::mt19937_64 r(7);
    long cases = 0, bad = 0;
    unsigned char s[32];
    auto check = [&]() {
        uint32_t u[8], h1, l1, n1, h2, l2, n2;
        std::memcpy(u, s, 32);
        rule(s, h1, l1, n1);
        ifa::packbits::pack32(u, h2, l2, n2);
        cases++;
        if (h1 != h2 || l1 != l2 || n1 != n2) bad++;
    };
    for (int pos = 0; pos < 32; pos++)
        for (int v = 0; v < 256; v++) {
            for (int i = 0; i < 32; i++) s[i] = "ACGTacgt"[r() & 7];
            s[pos] = static_cast<unsigned char>(v);
            check();
        }
    const char *alpha[] = {"ACGT", "acgtACGTnN", "ACGTNRYKMSWBDHV-*.acgtn"};
    for (long it = 0; it < 300000; it++) {
        const char *a = alpha[it % 3];
        const int n = static_cast<int>(std::strlen(a));
        for (int i = 0; i < 32; i++)
            s[i] = it % 5 == 0 ? static_cast<unsigned char>(r() & 0xff) : static_cast<unsigned char>(a[r() % n]);
        check();
    }
    std::printf("%ld %ld\n", cases, bad);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not found")
def test_pack32_matches_the_byte_rule(tmp_path):
    src = tmp_path / "pack_bits_test.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "pack_bits_test"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    cases, bad = int(out[0]), int(out[1])
    assert cases == 32 * 256 + 300000
    assert bad == 0
