"""Host check of the batched kernel's tile-row division (tile_row and
tile_row_magic in csrc/lbm_internal.cuh, shared by the host and the
kernel): floor(r / d) by one 64-bit multiply and a shift must equal integer
division for every divisor a tile width can take and every tile index of a
launch.  The header is compiled into a small host program by nvcc; no GPU
is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "lbm_internal.cuh"

static int check(int d, long long r, long long* bad) {
    unsigned m; int s;
    lbm::tile_row_magic(d, &m, &s);
    if (lbm::tile_row(static_cast<int>(r), m, s) != static_cast<int>(r / d)) { ++*bad; return 1; }
    return 0;
}

int main() {
    long long bad = 0, n = 0;
    uint64_t x = 0x9e3779b97f4a7c15ull;
    for (int d = 1; d <= 20000; ++d) {
        unsigned m; int s;
        lbm::tile_row_magic(d, &m, &s);
        // the multiplier's defining bounds: 2^s <= m d < 2^s + d, and m < 2^32
        const unsigned __int128 md = static_cast<unsigned __int128>(m) * d;
        const unsigned __int128 p = static_cast<unsigned __int128>(1) << s;
        if (md < p || md - p >= static_cast<unsigned __int128>(d)) ++bad;
        for (long long r = 0; r < 3ll * d + 3; ++r, ++n) check(d, r, &bad);
        for (int k = 0; k < 64; ++k, ++n) {
            x ^= x << 13; x ^= x >> 7; x ^= x << 17;
            check(d, static_cast<long long>(x & 0x7fffffffull), &bad);
        }
        const long long q = 0x7fffffffll / d;   // the last multiples below 2^31
        for (long long r = q * d - 2; r <= 0x7fffffffll && r <= q * d + 1; ++r, ++n)
            if (r >= 0) check(d, r, &bad);
    }
    const int big[] = {65536, 65537, 1 << 20, (1 << 20) + 1, 1 << 30, (1 << 30) + 7, 0x7fffffff};
    for (int d : big) {
        const long long rs[] = {0, 1, d - 1ll, static_cast<long long>(d), 0x7ffffffell, 0x7fffffffll};
        for (long long r : rs) { ++n; if (r >= 0 && r <= 0x7fffffffll) check(d, r, &bad); }
    }
    std::printf("%lld %lld\n", n, bad);
    return bad != 0;
}
"""


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_tile_row_equals_integer_division(tmp_path):
    cc = nvcc()
    if cc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "tile_row_check.cu"
    exe = tmp_path / "tile_row_check"
    src.write_text(PROGRAM)
    r = subprocess.run([cc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1412_7228_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    n, bad = (int(v) for v in out.stdout.split())
    assert out.returncode == 0 and bad == 0 and n > 10 ** 8, out.stdout
