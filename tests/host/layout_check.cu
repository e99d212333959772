// Host-side checks of the z layout and the polyphase order used by the
// framelet kernels for L >= 3 (compiled with nvcc, run on the CPU).
//
// Poly(nf, D) must be a bijection of 0..nf-1 that lists the positions of each
// residue class mod D in increasing order, class after class, and inv must
// undo pos.  z_index must map the (band, y, x) triples of every band to
// distinct positions inside the z buffer, with the 8 high-pass bands of a
// level contiguous per position and the positions 2^(l-1) apart of level l
// (L >= 3) next to each other.  Prints "ok" and exits 0 when every check
// holds; prints the first failure and exits 1 otherwise.
#include <cstdio>
#include <vector>

#include "../../paper_1504_07234_gb300/csrc/mlba_internal.cuh"

using mlba::Poly;
using mlba::z_index;

static int fail(const char* what, int a, int b, int c) {
  std::printf("FAIL %s %d %d %d\n", what, a, b, c);
  return 1;
}

int main() {
  const int sizes[] = {1, 2, 3, 5, 7, 8, 11, 16, 20, 37, 64, 70, 101, 1054, 4126};
  for (int nf : sizes) {
    for (int d = 1; d <= 8; d *= 2) {
      const Poly P(nf, d);
      // expected order: residue class a = 0..d-1, increasing inside a class
      int expect = 0;
      for (int a = 0; a < d; ++a) {
        if (P.start(a) != expect) return fail("start", nf, d, a);
        int cnt = 0;
        for (int x = a; x < nf; x += d) {
          if (P.pos(x) != expect) return fail("pos", nf, d, x);
          if (P.inv(expect) != x) return fail("inv", nf, d, x);
          ++expect;
          ++cnt;
        }
        if (P.count(a) != cnt) return fail("count", nf, d, a);
      }
      if (expect != nf) return fail("cover", nf, d, expect);
      int cmax = 0;
      for (int a = 0; a < d; ++a) cmax = P.count(a) > cmax ? P.count(a) : cmax;
      if (P.count_max() != cmax) return fail("count_max", nf, d, cmax);
    }
  }
  // z_index: a bijection of the band-major planes onto the z buffer
  const int zsizes[] = {5, 11, 20, 37};
  for (int nf : zsizes) {
    for (int levels = 1; levels <= 4; ++levels) {
      const int nb = 8 * levels + 1;
      const size_t plane = (size_t)nf * nf;
      std::vector<int> hit((size_t)nb * plane, 0);
      for (int b = 0; b < nb; ++b)
        for (int y = 0; y < nf; ++y)
          for (int x = 0; x < nf; ++x) {
            const size_t g = z_index(b, y, x, levels, nf);
            if (g >= hit.size()) return fail("z range", nf, levels, b);
            if (hit[g]++) return fail("z twice", nf, levels, b);
            // the high-pass bands of a level sit together per position
            if (b < nb - 1 && b % 8 != 0 && g != z_index(b - 1, y, x, levels, nf) + 1)
              return fail("z group", nf, levels, b);
            // the taps of level l, 2^(l-1) apart (L >= 3; 1 apart for L <= 2),
            // join neighbouring positions of the layout
            const int lev = b < nb - 1 ? b / 8 + 1 : levels;
            const int dl = levels >= 3 ? 1 << (lev - 1) : 1;
            const size_t step = b < nb - 1 ? 8 : 1;
            if (x + dl < nf && z_index(b, y, x + dl, levels, nf) != g + step)
              return fail("z dilation", nf, levels, b);
          }
      // L <= 2: the plain grouped layout
      if (levels <= 2 && z_index(nb - 1, 1, 2, levels, nf) != (size_t)(nb - 1) * plane + nf + 2)
        return fail("z plain", nf, levels, 0);
    }
  }
  std::printf("ok\n");
  return 0;
}
