"""Host-side checks of the K-block-major operand layouts (no GPU).

The index functions kblk_bf16 / kblk_e4m3 / kblk_f32 of the library's
internal header are compiled into a small host program with nvcc and
checked exhaustively on a few shapes (N a multiple of 128, rows odd and
even):

  * each is a bijection of [rows] x [N] onto [0, rows * N);
  * every TMA box (one K block of 64 BF16 / 128 E4M3 elements by box_rows
    rows, any row start) and every epilogue tile of kblk_f32 (128 pair
    elements by BN vectors) is one contiguous run, which is what the 3-D
    tensor maps and the tile stores assume;
  * the vector writers' element groups (pairs for the bfloat162 / float2
    accesses, eights for the E4M3 quantiser) stay adjacent.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "lgw_internal.cuh"
using namespace lgw;

template <class F>
static int check(const char *name, F idx, int rows, int N, int KB, int box_rows) {
  std::vector<char> seen((size_t)rows * N, 0);
  for (int r = 0; r < rows; ++r)
    for (int e = 0; e < N; ++e) {
      const size_t i = idx(r, e, rows);
      if (i >= seen.size() || seen[i]) { printf("%s: not a bijection at (%d,%d)\n", name, r, e); return 1; }
      seen[i] = 1;
    }
  // boxes: K block kb, rows r0 .. r0 + box_rows - 1 (r0 a multiple of box_rows)
  for (int kb = 0; kb < N / KB; ++kb)
    for (int r0 = 0; r0 + box_rows <= rows; r0 += box_rows) {
      const size_t base = idx(r0, kb * KB, rows);
      for (int r = 0; r < box_rows; ++r)
        for (int t = 0; t < KB; ++t)
          if (idx(r0 + r, kb * KB + t, rows) != base + (size_t)r * KB + t) {
            printf("%s: box (%d,%d) not contiguous\n", name, kb, r0); return 1;
          }
    }
  // element pairs and groups of eight stay adjacent
  for (int r = 0; r < rows; ++r)
    for (int e = 0; e < N; e += 8)
      for (int t = 1; t < 8; ++t)
        if (idx(r, e + t, rows) != idx(r, e, rows) + t) {
          printf("%s: group at (%d,%d) split\n", name, r, e); return 1;
        }
  return 0;
}

int main() {
  const int shapes[][2] = {{1, 128}, {7, 256}, {64, 384}, {130, 1024}};
  int bad = 0;
  for (auto &sh : shapes) {
    const int rows = sh[0], N = sh[1];
    for (int box : {1, 2, 64})
      if (box <= rows) {
        bad += check("kblk_bf16", [](int r, int e, int R) { return kblk_bf16(r, e, R); }, rows, N, 64, box);
        bad += check("kblk_e4m3", [](int r, int e, int R) { return kblk_e4m3(r, e, R); }, rows, N, 128, box);
        // kblk_f32 indexes (vector b, element e): a tile of 128 elements by box vectors
        bad += check("kblk_f32", [](int b, int e, int Bs) { return kblk_f32(b, e, Bs); }, rows, N, 128, box);
      }
  }
  printf(bad ? "FAIL\n" : "OK\n");
  return bad ? 1 : 0;
}
"""


def test_kblk_layouts_are_contiguous_bijections():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.cu")
        exe = os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write(PROGRAM)
        inc = ["-I", os.path.join(ROOT, "include"),
               "-I", os.path.join(ROOT, "paper_2310_20103_gb300", "csrc")]
        r = subprocess.run([nvcc, "-std=c++17", "-O1", *inc, src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout
