// Shared device helpers: complex and 3x3 colour algebra, lattice geometry,
// and the field accessors that hide the storage layouts.
//
// Layouts
//   canonical (the C ABI's, FP64): site-major arrays of complex128
//     U[V][4][9], W[V][8][9], vectors [V][ncomp]
//   packed (internal, FP32 / FP16): sites in groups of 16, each group storing
//     its sites' component planes one after another, element (site n, plane c)
//     of a field of npl planes at ((n / 16) npl + c) 16 + n % 16 ("AoSoA-16").
//     A warp reading one component of 16 consecutive sites touches one
//     contiguous run of 16 units, and the planes of one site lie a
//     compile-time distance apart, so a whole site is addressed from one base
//     pointer.  Every lattice extent is even, so V is a multiple of 16.
//     U: 4*9 planes, W: 8*9 planes, vectors: ncomp planes
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace swc {

// ------------------------------------------------------------------ complex
template <typename T> struct cx { T re, im; };

template <typename T> __device__ __forceinline__ cx<T> mk(T r, T i) { return {r, i}; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename T> __device__ __forceinline__ cx<T> cjmul(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename T> __device__ __forceinline__ cx<T> times_i(cx<T> a) { return {-a.im, a.re}; }
template <typename T> __device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }

template <typename T> struct V3 { cx<T> c[3]; };
template <typename T> struct M3 { cx<T> e[3][3]; };

template <typename T> __device__ __forceinline__ V3<T> zero3() {
  V3<T> v;
#pragma unroll
  for (int i = 0; i < 3; ++i) v.c[i] = {T(0), T(0)};
  return v;
}

// Complex multiply-accumulate a b into (re, im) with fused multiply-adds: 4
// per complex product (written out because a product formed first and then
// added costs 6: the compiler cannot fuse across the separate addition).
template <typename T> __device__ __forceinline__ void cmac(T& re, T& im, cx<T> a, cx<T> b) {
  re = fma(a.re, b.re, re);
  re = fma(-a.im, b.im, re);
  im = fma(a.re, b.im, im);
  im = fma(a.im, b.re, im);
}
// conj(a) b accumulated
template <typename T> __device__ __forceinline__ void cjmac(T& re, T& im, cx<T> a, cx<T> b) {
  re = fma(a.re, b.re, re);
  re = fma(a.im, b.im, re);
  im = fma(a.re, b.im, im);
  im = fma(-a.im, b.re, im);
}

// M v
template <typename T> __device__ __forceinline__ V3<T> mv(const M3<T>& M, const V3<T>& v) {
  V3<T> o;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T re = M.e[i][0].re * v.c[0].re, im = M.e[i][0].re * v.c[0].im;
    re = fma(-M.e[i][0].im, v.c[0].im, re);
    im = fma(M.e[i][0].im, v.c[0].re, im);
    cmac(re, im, M.e[i][1], v.c[1]);
    cmac(re, im, M.e[i][2], v.c[2]);
    o.c[i] = {re, im};
  }
  return o;
}
// M^+ v
template <typename T> __device__ __forceinline__ V3<T> mdv(const M3<T>& M, const V3<T>& v) {
  V3<T> o;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T re = M.e[0][i].re * v.c[0].re, im = M.e[0][i].re * v.c[0].im;
    re = fma(M.e[0][i].im, v.c[0].im, re);
    im = fma(-M.e[0][i].im, v.c[0].re, im);
    cjmac(re, im, M.e[1][i], v.c[1]);
    cjmac(re, im, M.e[2][i], v.c[2]);
    o.c[i] = {re, im};
  }
  return o;
}
template <typename T> __device__ __forceinline__ void acc3(V3<T>& a, const V3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i) a.c[i] = a.c[i] + b.c[i];
}
template <typename T> __device__ __forceinline__ void acc3s(V3<T>& a, T s, const V3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i) a.c[i] = a.c[i] + s * b.c[i];
}
template <typename T> __device__ __forceinline__ M3<T> mm(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T re = A.e[i][0].re * B.e[0][j].re, im = A.e[i][0].re * B.e[0][j].im;
      re = fma(-A.e[i][0].im, B.e[0][j].im, re);
      im = fma(A.e[i][0].im, B.e[0][j].re, im);
      cmac(re, im, A.e[i][1], B.e[1][j]);
      cmac(re, im, A.e[i][2], B.e[2][j]);
      C.e[i][j] = {re, im};
    }
  return C;
}
template <typename T> __device__ __forceinline__ M3<T> dag(const M3<T>& A) {
  M3<T> C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.e[i][j] = {A.e[j][i].re, -A.e[j][i].im};
  return C;
}
template <typename T> __device__ __forceinline__ void madd(M3<T>& A, const M3<T>& B) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A.e[i][j] = A.e[i][j] + B.e[i][j];
}

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];
  int stride[4];  // 1, L0, L0 L1, L0 L1 L2
  int V;
  int apbc;       // antiperiodic fermion BC in time
  int shape;      // site-block shape of the packed inner-precision fields (see site_shape), fixed per call
};

__host__ __device__ inline void coords(const Geom& g, int n, int x[4]) {
  x[0] = n % g.L[0];
  int q = n / g.L[0];
  x[1] = q % g.L[1];
  q /= g.L[1];
  x[2] = q % g.L[2];
  x[3] = q / g.L[2];
}

// neighbour index of n (coordinates x) one step `s` (+1/-1) along mu
__host__ __device__ inline int hop(const Geom& g, int n, const int x[4], int mu, int s) {
  if (s > 0) return (x[mu] == g.L[mu] - 1) ? n - (g.L[mu] - 1) * g.stride[mu] : n + g.stride[mu];
  return (x[mu] == 0) ? n + (g.L[mu] - 1) * g.stride[mu] : n - g.stride[mu];
}
// fermion boundary sign of a time hop from x3 in direction s
__device__ __forceinline__ bool bc_flip(const Geom& g, const int x[4], int s) {
  return g.apbc && ((s > 0) ? (x[3] == g.L[3] - 1) : (x[3] == 0));
}

// Blocked site order of the inner-precision (FP32/FP16) packed storage: the
// lattice is cut into blocks of B0 x B1 x B2 x B3 sites (powers of two),
// stored one after the other in lexicographic block order, the sites of a
// block contiguous in lexicographic order inside it.  A 128-site tile then
// covers a compact 4-D region, so more of a site's neighbours lie in the tile
// its block has just loaded.  The index is a sum of one term per direction,
// so a hop changes one term: n = sum_mu (b_mu bs_mu + l_mu ls_mu).
struct GeomBlk {
  int L[4];
  int lb[4];     // log2 B_mu
  int NB[4];     // blocks per direction
  int ls[4];     // stride of the in-block coordinate
  int bs[4];     // stride of the block coordinate (in sites)
  int V;
  int apbc;
};

// Site-block shapes (largest extents B0 x B1 x B2 x B3; shape 0 is the
// lexicographic order).  Each 128-site shape fills one reduction tile.
constexpr int kSiteShapes = 6;
__host__ __device__ inline void site_shape(int shape, int B[4]) {
  constexpr int kShapes[kSiteShapes][4] = {{1, 1, 1, 1}, {4, 4, 4, 2}, {8, 4, 2, 2},
                                           {8, 8, 2, 1}, {2, 4, 4, 4}, {4, 4, 2, 4}};
  const int k = (shape >= 0 && shape < kSiteShapes) ? shape : 0;
  for (int mu = 0; mu < 4; ++mu) B[mu] = kShapes[k][mu];
}

// Blocked geometry of `shape`: in each direction the block extent is the
// largest power of two up to the shape's that divides the lattice extent.
// shape 0 gives B = 1 everywhere, i.e. the lexicographic order.
__host__ __device__ inline GeomBlk make_blocked(const Geom& g, int shape) {
  GeomBlk b;
  int cap[4];
  site_shape(shape, cap);
  int bsz = 1;
  for (int mu = 0; mu < 4; ++mu) {
    int B = 1, lg = 0;
    while (B * 2 <= cap[mu] && g.L[mu] % (B * 2) == 0) {
      B *= 2;
      ++lg;
    }
    b.L[mu] = g.L[mu];
    b.lb[mu] = lg;
    b.NB[mu] = g.L[mu] >> lg;
    b.ls[mu] = bsz;
    bsz *= B;
  }
  int st = bsz;  // sites per block
  for (int mu = 0; mu < 4; ++mu) {
    b.bs[mu] = st;
    st *= b.NB[mu];
  }
  b.V = g.V;
  b.apbc = g.apbc;
  return b;
}

// blocked index of the site with coordinates x
__host__ __device__ inline int blk_index(const GeomBlk& g, const int x[4]) {
  int n = 0;
  for (int mu = 0; mu < 4; ++mu) {
    const int B = 1 << g.lb[mu];
    n += (x[mu] >> g.lb[mu]) * g.bs[mu] + (x[mu] & (B - 1)) * g.ls[mu];
  }
  return n;
}

__host__ __device__ inline void coords(const GeomBlk& g, int n, int x[4]) {
  // block index then in-block index, both lexicographic
  const int bsite = 1 << (g.lb[0] + g.lb[1] + g.lb[2] + g.lb[3]);
  int blk = n >> (g.lb[0] + g.lb[1] + g.lb[2] + g.lb[3]);
  int loc = n & (bsite - 1);
  for (int mu = 0; mu < 4; ++mu) {
    const int b = (mu < 3) ? blk % g.NB[mu] : blk;
    blk = (mu < 3) ? blk / g.NB[mu] : 0;
    const int B = 1 << g.lb[mu];
    const int l = loc & (B - 1);
    loc >>= g.lb[mu];
    x[mu] = (b << g.lb[mu]) + l;
  }
}

__host__ __device__ inline int hop(const GeomBlk& g, int n, const int x[4], int mu, int s) {
  const int B = 1 << g.lb[mu];
  const int l = x[mu] & (B - 1);
  if (s > 0) {
    if (l < B - 1) return n + g.ls[mu];
    n -= (B - 1) * g.ls[mu];
    return (x[mu] == g.L[mu] - 1) ? n - (g.NB[mu] - 1) * g.bs[mu] : n + g.bs[mu];
  }
  if (l > 0) return n - g.ls[mu];
  n += (B - 1) * g.ls[mu];
  return (x[mu] == 0) ? n + (g.NB[mu] - 1) * g.bs[mu] : n - g.bs[mu];
}

__device__ __forceinline__ bool bc_flip(const GeomBlk& g, const int x[4], int s) {
  return g.apbc && ((s > 0) ? (x[3] == g.L[3] - 1) : (x[3] == 0));
}

// Neighbour offsets of site n: n + df[mu] is the forward and n + db[mu] the
// backward neighbour along mu.  The site index is a sum of one term per
// direction (lexicographic and blocked orders alike), so a hop along mu
// changes only the mu-term and a diagonal neighbour -- a hypercube corner
// x + s -- is n plus one offset per direction.
template <typename GG>
__host__ __device__ inline void hop_deltas(const GG& g, int n, const int x[4], int df[4], int db[4]) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    df[mu] = hop(g, n, x, mu, +1) - n;
    db[mu] = hop(g, n, x, mu, -1) - n;
  }
}

// lexicographic site index -> blocked index (host and device)
__host__ __device__ inline int lex_to_blk(const GeomBlk& g, int n) {
  int x[4];
  x[0] = n % g.L[0];
  int q = n / g.L[0];
  x[1] = q % g.L[1];
  q /= g.L[1];
  x[2] = q % g.L[2];
  x[3] = q / g.L[2];
  return blk_index(g, x);
}

// ------------------------------------------------------------------ accessors
// Canonical FP64 (the C ABI layout)
struct GaugeC64 {
  static constexpr int kBytes = 4 * 9 * 16;  // per site
  static constexpr const char* kPrec = "f64";
  const double2* p;
  __device__ __forceinline__ M3<double> link(int n, int mu) const {
    const double2* q = p + ((size_t)n * 4 + mu) * 9;
    M3<double> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) { double2 v = __ldg(q + i * 3 + j); M.e[i][j] = {v.x, v.y}; }
    return M;
  }
};
struct TransC64 {
  static constexpr int kBytes = 8 * 9 * 16;
  const double2* p;
  __device__ __forceinline__ M3<double> mat(int n, int k) const {
    const double2* q = p + ((size_t)n * 8 + k) * 9;
    M3<double> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) { double2 v = __ldg(q + i * 3 + j); M.e[i][j] = {v.x, v.y}; }
    return M;
  }
};

// Packed (AoSoA-16) addressing: unit (site n, plane c) of a field of npl
// planes.  V is a multiple of 16 (even extents), so no group is partial.
__host__ __device__ __forceinline__ size_t pk(int n, int npl, int c) {
  return ((size_t)(n >> 4) * npl + c) * 16 + (n & 15);
}

// Packed FP32 links, 36 planes: plane mu*9 + 3i + j holds U_mu[i][j]
struct GaugeP32 {
  static constexpr int kBytes = 4 * 9 * 8;
  static constexpr const char* kPrec = "f32";
  const float2* p;
  __device__ __forceinline__ M3<float> link(int n, int mu) const {
    const float2* q = p + pk(n, 36, mu * 9);
    M3<float> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) { float2 v = __ldg(q + (i * 3 + j) * 16); M.e[i][j] = {v.x, v.y}; }
    return M;
  }
};
// Packed FP32 transports, 72 planes: plane k*9 + 3i + j holds W(x, s_k)[i][j]
struct TransP32 {
  static constexpr int kBytes = 8 * 9 * 8;
  const float2* p;
  __device__ __forceinline__ M3<float> mat(int n, int k) const {
    const float2* q = p + pk(n, 72, k * 9);
    M3<float> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) { float2 v = __ldg(q + (i * 3 + j) * 16); M.e[i][j] = {v.x, v.y}; }
    return M;
  }
};

// Vector fields: NC complex components per site.
template <int NC> struct VecC64 {  // canonical [V][NC] complex128
  using unit = double2;
  static size_t sys_units(int V) { return (size_t)V * NC; }
  double2* p;
  __device__ __forceinline__ cx<double> ld(int n, int c) const { double2 v = __ldg(p + (size_t)n * NC + c); return {v.x, v.y}; }
  __device__ __forceinline__ void st(int n, int c, cx<double> a) const { p[(size_t)n * NC + c] = make_double2(a.re, a.im); }
};
template <int NC> struct VecP32 {  // packed, NC float2 planes
  using unit = float2;
  static size_t sys_units(int V) { return (size_t)V * NC; }
  float2* p;
  int V;  // volume (the packed addressing itself needs only n)
  __device__ __forceinline__ cx<float> ld(int n, int c) const { float2 v = __ldg(p + pk(n, NC, c)); return {v.x, v.y}; }
  __device__ __forceinline__ void st(int n, int c, cx<float> a) const { p[pk(n, NC, c)] = make_float2(a.re, a.im); }
};

// Packed FP32 with two complex components per 16-byte unit: NC/2 float4
// planes, plane k holding components (2k, 2k+1).  Whole-site loads and stores
// use half as many, twice as wide, memory instructions (NC even).
template <int NC> struct VecP32q {
  static_assert(NC % 2 == 0, "pairs of components");
  using unit = float4;
  static size_t sys_units(int V) { return (size_t)V * NC / 2; }
  float4* p;
  int V;  // volume (the packed addressing itself needs only n)
  __device__ __forceinline__ cx<float> ld(int n, int c) const {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p + pk(n, NC / 2, c >> 1)) + (c & 1));
    return {v.x, v.y};
  }
  __device__ __forceinline__ void st(int n, int c, cx<float> a) const {
    reinterpret_cast<float2*>(p + pk(n, NC / 2, c >> 1))[c & 1] = make_float2(a.re, a.im);
  }
};

// Packed FP32 vectors of pairs of systems: systems 2k and 2k+1 share pair k,
// whose unit (site n, component c) holds (s0.re, s1.re, s0.im, s1.im), so one
// 16-byte load gives both systems' component as the lanes of two float2
// registers -- the operands of two-lane arithmetic over a pair of systems,
// with no regrouping.  An accessor is one system's view: the pair's base and
// the system's lane.  A system's share of a pair is sys_units (half a pair);
// batches allocate whole pairs.
template <int NC> struct VecP32x2 {
  using unit = float4;
  static constexpr bool kPaired = true;
  static size_t sys_units(int V) { return (size_t)V * NC / 2; }
  float4* p;
  int V;  // volume (the packed addressing itself needs only n)
  int lane = 0;
  __device__ __forceinline__ cx<float> ld(int n, int c) const {
    const float* q = reinterpret_cast<const float*>(p + pk(n, NC, c));
    return {__ldg(q + lane), __ldg(q + 2 + lane)};
  }
  __device__ __forceinline__ void st(int n, int c, cx<float> a) const {
    float* q = reinterpret_cast<float*>(p + pk(n, NC, c));
    q[lane] = a.re;
    q[2 + lane] = a.im;
  }
};
template <class V, class = void> struct is_paired : std::false_type {};
template <class V> struct is_paired<V, std::void_t<decltype(V::kPaired)>> : std::bool_constant<V::kPaired> {};

// Packed two-lane FP32 arithmetic (one f32x2 instruction for two FP32
// operations; an operand used in both lanes is broadcast).
// (The library is built for sm_103a only; the lane-by-lane forms exist so that
// host-side tests that include this header compile for the default arch.)
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
#if !defined(__CUDA_ARCH__) || __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
#else
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
#endif

// Packed FP16 storage (mixed precision "half" mode; arithmetic stays FP32).
//   links: the first two rows only (12 reals) as 6 half2 planes per direction
//          (24 planes); the third row is rebuilt as conj(row0 x row1), exact
//          for SU(3) links
//   transports: all 9 entries, 72 half2 planes (not unitary: no compression)
//   vectors: NC half2 planes holding psi/scale, then one float scale per site
//          (the largest |re|, |im| of the site, site-major), so every site
//          keeps FP16's relative precision whatever its magnitude
__device__ __forceinline__ cx<float> h2c(__half2 h) {
  const float2 f = __half22float2(h);
  return {f.x, f.y};
}

// row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1)
__device__ __forceinline__ void su3_third_row(M3<float>& M) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int a = (j + 1) % 3, b = (j + 2) % 3;
    // c = row0_a row1_b - row0_b row1_a, as fused multiply-adds
    float re = M.e[0][a].re * M.e[1][b].re, im = M.e[0][a].re * M.e[1][b].im;
    re = fma(-M.e[0][a].im, M.e[1][b].im, re);
    im = fma(M.e[0][a].im, M.e[1][b].re, im);
    re = fma(-M.e[0][b].re, M.e[1][a].re, re);
    re = fma(M.e[0][b].im, M.e[1][a].im, re);
    im = fma(-M.e[0][b].re, M.e[1][a].im, im);
    im = fma(-M.e[0][b].im, M.e[1][a].re, im);
    M.e[2][j] = {re, -im};
  }
}

struct GaugeP16 {
  static constexpr int kBytes = 4 * 6 * 4;
  static constexpr const char* kPrec = "f16";
  const __half2* p;
  __device__ __forceinline__ M3<float> link(int n, int mu) const {
    const __half2* q = p + pk(n, 24, mu * 6);
    M3<float> M;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M.e[i][j] = h2c(__ldg(q + (i * 3 + j) * 16));
    su3_third_row(M);
    return M;
  }
};
struct TransP16 {
  static constexpr int kBytes = 8 * 9 * 4;
  const __half2* p;
  __device__ __forceinline__ M3<float> mat(int n, int k) const {
    const __half2* q = p + pk(n, 72, k * 9);
    M3<float> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M.e[i][j] = h2c(__ldg(q + (i * 3 + j) * 16));
    return M;
  }
};
template <int NC> struct VecP16 {  // per system: NC packed half2 planes, then [V] float scales
  using unit = __half2;
  static size_t sys_units(int V) { return (size_t)V * (NC + 1); }
  __half2* p;
  int V;
  __device__ __forceinline__ const float* sc() const { return reinterpret_cast<const float*>(p + (size_t)NC * V); }
  __device__ __forceinline__ cx<float> ld(int n, int c) const {
    const cx<float> v = h2c(__ldg(p + pk(n, NC, c)));
    const float s = __ldg(sc() + n);
    return {v.re * s, v.im * s};
  }
};

template <typename Acc, typename T> __device__ __forceinline__ V3<T> ld3(const Acc& a, int n, int off = 0) {
  V3<T> v;
#pragma unroll
  for (int i = 0; i < 3; ++i) v.c[i] = a.ld(n, off + i);
  return v;
}

// ------------------------------------------------------------------ reductions
// Block-wide sum of one double per thread (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* smem /* >= 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) smem[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = (lane < nw) ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

}  // namespace swc
