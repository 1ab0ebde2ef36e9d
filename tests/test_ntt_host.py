"""The acquisition transform's index arithmetic on the host (no GPU).

rx_ntt.cuh's pass routines are host/device: here a small C++ program runs them
thread by thread, pass by pass, in the row kernel's schedule (forward: a radix-2 pass
where the shared-memory stage count is odd, radix-4 passes, the 32-element register
pass; inverse: the register pass, dit_middle's radix-16 and radix-4 passes, the
last pass that keeps the outputs below M / 2), for every transform size the
acquisition supports (2^11 .. 2^15) with the kernel's thread counts.  The result
must be the cyclic convolution of the two inputs over GF(2^30 - 2^18 + 1), checked
against the direct sum at every kept output for 2^11 and at 64 random kept outputs
for the larger sizes; the program also checks that no pass touches an element
outside the transform.  Twiddles are built here from their definition
(w_{2L} = 11^((p - 1) / (2L))), not taken from the library."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_00463_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>
#include <random>
#include "rx_ntt.cuh"
using namespace rxn;
static const uint64_t P = kP;
static uint64_t pw(uint64_t b, uint64_t e) { uint64_t r = 1; b %= P; while (e) { if (e & 1) r = r * b % P; b = b * b % P; e >>= 1; } return r; }
static uint2 wq(uint32_t w) { uint2 t; t.x = w; t.y = (uint32_t)(((uint64_t)w << 32) / P); return t; }
struct TabF { const uint2 *t; uint2 operator[](int k) const { return t[k]; } };
int main() {
    const uint32_t NMAX = 1u << kMaxLog;
    std::vector<uint2> T(NMAX), Ti(NMAX);
    for (uint32_t L = 1; L < NMAX; L *= 2) {
        uint64_t w = pw(kGen, (P - 1) / (2 * L)), wi = pw(w, P - 2), a = 1, b = 1;
        for (uint32_t j = 0; j < L; ++j) { T[L + j] = wq((uint32_t)a); Ti[L + j] = wq((uint32_t)b); a = a * w % P; b = b * wi % P; }
    }
    std::mt19937_64 rng(463100);
    int bad = 0;
    for (int logM = 11; logM <= 15; ++logM) {
        const uint32_t M = 1u << logM, NT = logM >= 14 ? 512u : M / 32, W = M + M / 8;
        const int RL = 5, R = 32;
        std::vector<uint32_t> x(M), y(M);
        for (uint32_t i = 0; i < M; ++i) { x[i] = (uint32_t)(rng() % P); y[i] = (uint32_t)(rng() % P); }
        // padded buffers with guard words that no pass may touch
        const uint32_t G = 64, GUARD = 0xdeadbeefu;
        auto fwd = [&](const std::vector<uint32_t> &in) {
            std::vector<uint32_t> buf(W + 2 * G, GUARD);
            uint32_t *s = buf.data() + G;
            for (uint32_t i = 0; i < M; ++i) s[pad(i)] = in[i];
            int lg = logM - 1;
            if (smem_stages(logM, RL) & 1) { for (uint32_t t = 0; t < NT; ++t) dif_pass2(s, lg, t, NT, M, T.data()); lg -= 1; }
            for (; lg >= RL + 1; lg -= 2) for (uint32_t t = 0; t < NT; ++t) dif_pass4(s, lg - 1, t, NT, M, T.data());
            for (uint32_t q = 0; q < M / R; ++q) {
                uint32_t v[32];
                for (int e = 0; e < R; ++e) v[e] = s[pad(R * q + e)];
                dif_reg<5>(v, TabF{T.data()});
                for (int e = 0; e < R; ++e) s[pad(R * q + e)] = v[e];
            }
            for (uint32_t k = 0; k < G; ++k) if (buf[k] != GUARD || buf[G + W + k] != GUARD) { std::printf("guard hit fwd %d\n", logM); std::exit(1); }
            std::vector<uint32_t> out(M);
            for (uint32_t i = 0; i < M; ++i) out[i] = s[pad(i)];
            return out;
        };
        std::vector<uint32_t> X = fwd(x), Y = fwd(y);
        const uint64_t minv = pw(M, P - 2);
        std::vector<uint32_t> buf(W + 2 * G, GUARD);
        uint32_t *s = buf.data() + G;
        for (uint32_t i = 0; i < M; ++i) s[pad(i)] = shoup(X[i], wq((uint32_t)(Y[i] % P * minv % P)));
        for (uint32_t q = 0; q < M / R; ++q) {
            uint32_t v[32];
            for (int e = 0; e < R; ++e) v[e] = s[pad(R * q + e)];
            dit_reg<5>(v, TabF{Ti.data()});
            for (int e = 0; e < R; ++e) s[pad(R * q + e)] = v[e];
        }
        for (int p = 0; p < dit_middle_count(logM, RL); ++p)
            for (uint32_t t = 0; t < NT; ++t) dit_middle_pass(p, s, logM, RL, t, NT, Ti.data());
        for (uint32_t k = 0; k < G; ++k) if (buf[k] != GUARD || buf[G + W + k] != GUARD) { std::printf("guard hit inv %d\n", logM); std::exit(1); }
        std::vector<int64_t> got(M / 2, INT64_MIN);
        auto sink = [&](uint32_t, uint32_t c, int32_t z) { if (c < M / 2) got[c] = z; };
        // the last pass reads the buffer only; run it for every thread
        switch (logM) {
            case 11: for (uint32_t t = 0; t < NT; ++t) LastHalf<11, 64, 5>::run(s, t, Ti.data(), sink); break;
            case 12: for (uint32_t t = 0; t < NT; ++t) LastHalf<12, 128, 5>::run(s, t, Ti.data(), sink); break;
            case 13: for (uint32_t t = 0; t < NT; ++t) LastHalf<13, 256, 5>::run(s, t, Ti.data(), sink); break;
            case 14: for (uint32_t t = 0; t < NT; ++t) LastHalf<14, 512, 5>::run(s, t, Ti.data(), sink); break;
            default: for (uint32_t t = 0; t < NT; ++t) LastHalf<15, 512, 5>::run(s, t, Ti.data(), sink); break;
        }
        std::vector<uint32_t> idx;
        if (logM == 11) for (uint32_t c = 0; c < M / 2; ++c) idx.push_back(c);
        else for (int k = 0; k < 64; ++k) idx.push_back((uint32_t)(rng() % (M / 2)));
        for (uint32_t c : idx) {
            uint64_t acc = 0;
            for (uint32_t k = 0; k < M; ++k) acc = (acc + (uint64_t)x[k] * y[(c + M - k) % M]) % P;
            int64_t want = acc > (P - 1) / 2 ? (int64_t)acc - (int64_t)P : (int64_t)acc;
            if (got[c] != want) { if (bad < 5) std::printf("M=2^%d c=%u got %lld want %lld\n", logM, c, (long long)got[c], (long long)want); ++bad; }
        }
        for (uint32_t c = 0; c < M / 2; ++c) if (got[c] == INT64_MIN) { std::printf("M=2^%d output %u not produced\n", logM, c); ++bad; break; }
    }
    if (bad) { std::printf("%d mismatches\n", bad); return 1; }
    std::printf("ok\n");
    return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("ntt")
    src, exe = d / "ntt_harness.cpp", d / "ntt_harness"
    src.write_text(HARNESS)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_transform_passes_compute_the_cyclic_convolution(harness):
    r = subprocess.run([str(harness)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
