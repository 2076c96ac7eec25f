"""Host-side layout of the staged Neumann sweeps (stage_layout) and the stencil-pattern
classification (stencil_pattern), compiled with nvcc into a small host program and run
without a GPU.  For every trip of every block the program walks the windows the sweep
copies and the shared-memory reads it makes (the same index arithmetic as the kernel:
two quads of four rows per thread, R = 8 x threads rows per trip) and checks that every
bulk copy is 16-byte aligned, whole 16-byte groups, inside the vector and inside its part
of the stage, that every read stays inside the stage, and that two stages fit beside the
kernel's static shared memory."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SOURCE = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "common.cuh"
using namespace pbcg;

#define REQUIRE(c) do { if (!(c)) { printf("FAIL %s line %d: %s\n", name, __LINE__, #c); return 1; } } while (0)

// Walk one configuration: n rows, the ascending offsets, threads per block, grid blocks,
// chunked or grid-stride row order (chunk rounded to 4 as the four-row kernels do).
static int walk(const char* name, int n, const std::vector<int>& off, int threads, int grid, bool strided,
                bool expect_ok) {
  StageLayout L;
  const int R = 8 * threads;
  stage_layout(L, off.data(), (int)off.size(), R);
  REQUIRE(L.ok == (expect_ok ? 1 : 0));
  if (!L.ok) return 0;
  REQUIRE(L.H % 4 == 0 && L.H >= 4 && L.R == R);
  const int nearw = R + 2 * L.H;
  REQUIRE(L.mask_f % 4 == 0 && L.stage_f % 4 == 0 && L.stage_f == L.mask_f + (R + 8) / 2);
  REQUIRE(2LL * L.stage_f * 4 + 4752 <= 232448);   // two stages + the kernel's static shared memory
  const int nmask = ((n + 7) & ~7) + 8;
  int chunk = (n + grid - 1) / grid;
  chunk = (chunk + 3) / 4 * 4;
  for (int b = 0; b < grid; ++b) {
    const int first = strided ? 8 * b * threads : std::min(n, b * chunk);
    const int stride = strided ? 8 * grid * threads : 8 * threads;
    const int end = strided ? n : std::min(n, b * chunk + chunk);
    for (int base = first; base < end; base += stride) {
      REQUIRE(base % 4 == 0);
      long long tx = 0;
      auto win = [&](int dst, int lo, int cnt, int part_end) {
        const int a0 = std::max(lo, 0), a1 = std::min(lo + cnt, n);
        if (a1 <= a0) return true;
        if (a0 % 4 || a1 % 4 || (dst + a0 - lo) % 4) return false;              // 16-byte groups
        if (dst + (a0 - lo) < 0 || dst + (a1 - lo) > part_end) return false;    // inside its part
        tx += 4LL * (a1 - a0);
        return true;
      };
      REQUIRE(win(0, base - L.H, nearw, nearw));
      for (int f = 0; f < L.nfar; ++f) REQUIRE(win(nearw + f * R, base + L.far[f], R, nearw + (f + 1) * R));
      const int mlo = base & ~7, mhi = std::min(mlo + R + 8, nmask);
      REQUIRE(mlo % 8 == 0 && mhi % 8 == 0 && mhi > mlo);
      REQUIRE(2 * L.mask_f + (mhi - mlo) <= 2 * L.stage_f);
      tx += 2LL * (mhi - mlo);
      REQUIRE(tx < (1 << 20) - 1);                                              // mbarrier tx-count
      for (int q = 0; q < 2; ++q)
        for (int t : {0, threads - 1}) {
          const int qo = q * 4 * threads, own = L.H + qo + 4 * t;
          REQUIRE(own - 3 >= 0 && own + 6 < nearw);                             // +-3 rows around the quad
          for (size_t d = 0; d < off.size(); ++d) {
            const int o = off[d];
            if (o >= -3 && o <= 3) continue;
            int sb = L.H + o, lim = nearw;
            if (o < -R || o > R) {
              int f = 0;
              while (f < L.nfar - 1 && L.far[f] != o) ++f;
              REQUIRE(L.far[f] == o);
              sb = nearw + f * R;
              lim = sb + R;
            }
            REQUIRE(sb + qo + 4 * t >= 0 && sb + qo + 4 * t + 3 < lim);
          }
          const int mrow = 2 * L.mask_f + (base - mlo) + qo + 4 * t;
          REQUIRE(mrow % 4 == 0 && mrow + 3 < 2 * L.stage_f);
        }
    }
  }
  return 0;
}

int main() {
  const char* name = "pattern";
  {
    const int p3[] = {-65536, -256, -1, 0, 1, 256, 65536}, p3t[] = {-65536, -256, -1, 1, 256, 65536};
    const int p2[] = {-1024, -1, 0, 1, 1024}, p2t[] = {-1024, -1, 1, 1024};
    const int odd[] = {-130, -1, 0, 1, 130}, wide[] = {-1024, -2, 0, 2, 1024}, six[] = {-8, -4, -1, 0, 1, 4};
    REQUIRE(stencil_pattern(p3, 7) == 7 && stencil_pattern(p3t, 6) == 6);
    REQUIRE(stencil_pattern(p2, 5) == 5 && stencil_pattern(p2t, 4) == 4);
    REQUIRE(stencil_pattern(odd, 5) == 0 && stencil_pattern(wide, 5) == 0 && stencil_pattern(six, 6) == 0);
  }
  auto o3 = [](int N) { return std::vector<int>{-N * N, -N, -1, 0, 1, N, N * N}; };
  auto o2 = [](int N) { return std::vector<int>{-N, -1, 0, 1, N}; };
  if (walk("3d_256_768", 256 * 256 * 256, o3(256), 768, 152, true, true)) return 1;
  if (walk("3d_160_768", 160 * 160 * 160, o3(160), 768, 152, true, true)) return 1;
  if (walk("3d_40_512", 64000, o3(40), 512, 125, true, true)) return 1;
  if (walk("3d_40_128", 64000, o3(40), 128, 500, true, true)) return 1;
  if (walk("3d_34_64", 34 * 34 * 34, o3(34), 64, 608, true, true)) return 1;
  if (walk("2d_130_32", 130 * 130, o2(130), 32, 528, true, true)) return 1;
  if (walk("2d_262_32", 262 * 262, o2(262), 32, 1216, true, false)) return 1;   // far and unaligned
  if (walk("2d_512_512", 512 * 512, o2(512), 512, 152, false, true)) return 1;  // chunked
  if (walk("2d_1024_512", 1024 * 1024, o2(1024), 512, 152, false, true)) return 1;
  printf("ok\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def nvcc():
    from paper_1809_01948_gb300._build import _nvcc
    return _nvcc()


def test_staged_layout_bounds_and_patterns(nvcc):
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.cu"), os.path.join(d, "layout")
        open(src, "w").write(SOURCE)
        subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                               "arch=compute_103a,code=sm_103a",
                               "-I", os.path.join(ROOT, "paper_1809_01948_gb300", "csrc"),
                               "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), (out.returncode, out.stdout, out.stderr)
