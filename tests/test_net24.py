"""The 24-position sorting network of the setup kernels (csrc/net24.cuh), on
the CPU: the header compiles as plain C++, and the pruned odd-even merge
network it defines sorts every input. By the 0-1 principle (a comparator
network sorts every input if and only if it sorts every sequence of 0s and 1s)
it suffices to run all 2^24 such sequences, which the check does bit-sliced
(64 sequences per machine word). The thread-per-row proposal ordering and row
products sort their rows with this network."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1806_07028_gb300", "csrc")

CHECK = r"""
#include <cstdint>
#include <cstdio>
#include <vector>
#include "net24.cuh"

int main() {
    using pc::kNet24;
    using pc::kNet24Size;
    using pc::net24;
    for (int q = 0; q < kNet24Size; ++q) {
        const int a = net24(q, true), c = net24(q, false);
        if (!(0 <= a && a < c && c < kNet24)) { std::printf("comparator %d: %d %d\n", q, a, c); return 1; }
    }
    // position p of sequence s holds bit p of s; word w holds sequences 64w .. 64w + 63
    const size_t W = (size_t)1 << (kNet24 - 6);
    const uint64_t low[6] = {0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
                             0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};
    std::vector<uint64_t> X((size_t)kNet24 * W);
    for (int p = 0; p < kNet24; ++p)
        for (size_t w = 0; w < W; ++w)
            X[p * W + w] = p < 6 ? low[p] : (((w >> (p - 6)) & 1) ? ~0ull : 0ull);
    for (int q = 0; q < kNet24Size; ++q) {   // min to the lower position, max to the upper
        uint64_t* xa = &X[net24(q, true) * W];
        uint64_t* xc = &X[net24(q, false) * W];
        for (size_t w = 0; w < W; ++w) {
            const uint64_t lo = xa[w] & xc[w], hi = xa[w] | xc[w];
            xa[w] = lo;
            xc[w] = hi;
        }
    }
    for (int p = 0; p + 1 < kNet24; ++p)
        for (size_t w = 0; w < W; ++w)
            if (X[p * W + w] & ~X[(p + 1) * W + w]) { std::printf("unsorted at %d, word %zu\n", p, w); return 1; }
    std::printf("ok %d\n", kNet24Size);
    return 0;
}
"""


def _run(tmp_path, src):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    c = tmp_path / "check.cpp"
    c.write_text(src)
    exe = tmp_path / "check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, str(c), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True)


def test_net24_sorts_every_input(tmp_path):
    r = _run(tmp_path, CHECK)
    assert r.returncode == 0, r.stdout
    assert r.stdout.strip() == "ok 132"


def test_check_catches_a_network_missing_a_comparator(tmp_path):
    # the same check with one comparator dropped must find an unsorted input
    src = CHECK.replace("for (int q = 0; q < kNet24Size; ++q) {   // min",
                        "for (int q = 1; q < kNet24Size; ++q) {   // min")
    assert src != CHECK
    r = _run(tmp_path, src)
    assert r.returncode == 1 and r.stdout.startswith("unsorted")
