// Host-side check of the site addressing used by the stencils (common.cuh,
// dslash.cuh): the blocked site order is a permutation of the sites, coords()
// inverts blk_index(), and a hop in the blocked order lands on the blocked
// index of the lexicographic neighbour, for every site, direction and sign
// (periodic wrap included); the per-site offsets reach all 16 hypercube
// corners x +- s in both orders; the packed (AoSoA-16) unit index is a
// bijection.  Every site-block shape of the menu, on lattices whose extents
// the shapes divide and do not divide.  Prints "ok" or the first mismatch.
#include <cstdio>
#include <vector>

#include "../../paper_1312_3265_gb300/csrc/common.cuh"
#include "../../paper_1312_3265_gb300/csrc/dslash.cuh"

using namespace swc;

static int check(int L0, int L1, int L2, int L3, int shape) {
  Geom g;
  g.L[0] = L0; g.L[1] = L1; g.L[2] = L2; g.L[3] = L3;
  g.stride[0] = 1; g.stride[1] = L0; g.stride[2] = L0 * L1; g.stride[3] = L0 * L1 * L2;
  g.V = L0 * L1 * L2 * L3;
  g.apbc = 0;
  g.shape = shape;
  const GeomBlk b = make_blocked(g, shape);
  std::vector<int> seen(g.V, 0);
  for (int n = 0; n < g.V; ++n) {
    int x[4] = {n % L0, (n / L0) % L1, (n / (L0 * L1)) % L2, n / (L0 * L1 * L2)};
    const int nb = lex_to_blk(b, n);
    if (nb < 0 || nb >= g.V || seen[nb]++) { printf("not a permutation at %d (%dx%dx%dx%d)\n", n, L0, L1, L2, L3); return 1; }
    int y[4];
    coords(b, nb, y);
    for (int mu = 0; mu < 4; ++mu)
      if (y[mu] != x[mu]) { printf("coords mismatch at %d\n", n); return 1; }
    for (int mu = 0; mu < 4; ++mu)
      for (int s = -1; s <= 1; s += 2) {
        int z[4] = {x[0], x[1], x[2], x[3]};
        z[mu] = (z[mu] + s + g.L[mu]) % g.L[mu];
        const int want = blk_index(b, z);
        const int got = hop(b, nb, x, mu, s);
        if (got != want) { printf("hop mismatch n=%d mu=%d s=%d (%dx%dx%dx%d)\n", n, mu, s, L0, L1, L2, L3); return 1; }
      }
  }
  // hypercube corners from per-site offsets (lexicographic and blocked order)
  for (int n = 0; n < g.V; ++n) {
    int x[4] = {n % L0, (n / L0) % L1, (n / (L0 * L1)) % L2, n / (L0 * L1 * L2)};
    const int nb = lex_to_blk(b, n);
    int df[4], db[4], bf[4], bb[4];
    hop_deltas(g, n, x, df, db);
    hop_deltas(b, nb, x, bf, bb);
    for (int k = 0; k < 8; ++k) {
      int zf[4], zb[4];
      for (int mu = 0; mu < 4; ++mu) {
        const int s = (mu == 3) ? 1 : (((k >> mu) & 1) ? -1 : 1);
        zf[mu] = (x[mu] + s + g.L[mu]) % g.L[mu];
        zb[mu] = (x[mu] - s + g.L[mu]) % g.L[mu];
      }
      const int lf = zf[0] + L0 * (zf[1] + L1 * (zf[2] + L2 * zf[3]));
      const int lb = zb[0] + L0 * (zb[1] + L1 * (zb[2] + L2 * zb[3]));
      int of, ob;
      corner_offsets(k, df, db, of, ob);
      if (n + of != lf || n + ob != lb) { printf("corner mismatch n=%d k=%d (%dx%dx%dx%d)\n", n, k, L0, L1, L2, L3); return 1; }
      corner_offsets(k, bf, bb, of, ob);
      if (nb + of != blk_index(b, zf) || nb + ob != blk_index(b, zb)) {
        printf("blocked corner mismatch n=%d k=%d (%dx%dx%dx%d)\n", n, k, L0, L1, L2, L3);
        return 1;
      }
    }
  }
  if (shape != 1) return 0;
  // packed unit index: a bijection of (site, plane) onto [0, V npl)
  for (int npl : {3, 6, 12, 24, 36, 72}) {
    std::vector<char> hit((size_t)g.V * npl, 0);
    for (int n = 0; n < g.V; ++n)
      for (int c = 0; c < npl; ++c) {
        const size_t i = pk(n, npl, c);
        if (i >= hit.size() || hit[i]++) { printf("packed index clash npl=%d n=%d c=%d\n", npl, n, c); return 1; }
      }
  }
  return 0;
}

int main() {
  const int dims[][4] = {{2, 2, 2, 2}, {4, 4, 4, 4}, {6, 6, 4, 6}, {16, 16, 16, 32}, {2, 4, 6, 2}, {10, 4, 6, 10},
                         {24, 24, 24, 48}, {12, 12, 12, 24}, {8, 8, 8, 8}};
  for (auto& d : dims)
    for (int shape = 0; shape < kSiteShapes; ++shape)
      if (check(d[0], d[1], d[2], d[3], shape)) {
        printf("(site-block shape %d)\n", shape);
        return 1;
      }
  printf("ok\n");
  return 0;
}
