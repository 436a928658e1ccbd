// Wilson operator: FP64 apply (C ABI) and batched CGNE.  r = 1 uses the
// spin-projected hop, other r the full 4-spinor hop.
#include "driver.cuh"

namespace swc {

template <bool R1> using W64 = WOp<double, GaugeC64, VecC64, R1>;
template <bool R1> using W32 = WOp<float, GaugeP32, VecP32q, R1>;
using W32L = WOp<float, GaugeP32, VecP32q, true, true>;  // the lean r = 1 form
template <bool R1> using W16 = WOp<float, GaugeP16, VecP16, R1>;

template <bool R1>
static int apply_impl(const Geom& g, const double2* U, const double2* in, double2* out, double mass, double r,
                      int dagger, cudaStream_t st) {
  const W64<R1> op{GaugeC64{U}};
  const int gx = (g.V + 127) / 128;
  apply_kernel<double, W64<R1>><<<dim3(gx, 1), 128, 0, st>>>(g, op, VecC64<12>{const_cast<double2*>(in)},
                                                             VecC64<12>{out}, mass, 0, r, dagger,
                                                             nullptr, 0);
  note_launches(1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SW_OK : cuda_fail(e);
}

int wilson_apply_f64(const Geom& g, const double2* U, const double2* in, double2* out, double mass, double r,
                     int dagger, cudaStream_t st) {
  return (r == 1.0) ? apply_impl<true>(g, U, in, out, mass, r, dagger, st)
                    : apply_impl<false>(g, U, in, out, mass, r, dagger, st);
}

template <bool R1>
static int cgne_impl(const Geom& g, const SolveArgs& a) {
  const W64<R1> opd{GaugeC64{a.U}};
  if (a.precision == SW_PREC_F64) return run_cgne<W64<R1>, W64<R1>, false>(g, opd, opd, a);
  if (a.precision == SW_PREC_F32_RELIABLE) {
    DevMem mu;
    if (!mu.alloc(sizeof(float2) * 36 * (size_t)g.V, a.stream)) return SW_ERR_OOM;
    pack_mats_p32<<<sm_count() * 8, 256, 0, a.stream>>>(make_blocked(g, g.shape), 4, a.U, mu.as<float2>());
    note_launches(1);
    if constexpr (R1)
      if (wilson_lean(g)) return run_cgne<W64<R1>, W32L, true>(g, opd, W32L{GaugeP32{mu.as<float2>()}}, a);
    const W32<R1> opf{GaugeP32{mu.as<float2>()}};
    return run_cgne<W64<R1>, W32<R1>, true>(g, opd, opf, a);
  }
  if (a.precision == SW_PREC_F16_RELIABLE) {
    if (int e = check_su3(g, a.U, a.stream)) return e;
    DevMem mu;
    if (!mu.alloc(sizeof(__half2) * 24 * (size_t)g.V, a.stream)) return SW_ERR_OOM;
    pack_links_h12<<<sm_count() * 8, 256, 0, a.stream>>>(make_blocked(g, g.shape), a.U, mu.as<__half2>());
    note_launches(1);
    const W16<R1> opf{GaugeP16{mu.as<__half2>()}};
    return run_cgne<W64<R1>, W16<R1>, true>(g, opd, opf, a);
  }
  return SW_ERR_ARG;
}

int wilson_cgne(const Geom& g, const SolveArgs& a) {
  return (a.r == 1.0) ? cgne_impl<true>(g, a) : cgne_impl<false>(g, a);
}


template <bool R1>
static int inner_impl(const Geom& g, const double2* U, const double2* in, double2* out, int nsys,
                      const double* masses, double r, int dagger, int precision, cudaStream_t st) {
  if (precision == SW_PREC_F32_RELIABLE) {
    DevMem mu;
    if (!mu.alloc(sizeof(float2) * 36 * (size_t)g.V, st)) return SW_ERR_OOM;
    pack_mats_p32<<<sm_count() * 8, 256, 0, st>>>(make_blocked(g, g.shape), 4, U, mu.as<float2>());
    note_launches(1);
    if constexpr (R1)
      if (wilson_lean(g)) return run_inner_apply(g, W32L{GaugeP32{mu.as<float2>()}}, in, out, nsys, masses, r, dagger, st);
    return run_inner_apply(g, W32<R1>{GaugeP32{mu.as<float2>()}}, in, out, nsys, masses, r, dagger, st);
  }
  if (precision == SW_PREC_F16_RELIABLE) {
    if (int e = check_su3(g, U, st)) return e;
    DevMem mu;
    if (!mu.alloc(sizeof(__half2) * 24 * (size_t)g.V, st)) return SW_ERR_OOM;
    pack_links_h12<<<sm_count() * 8, 256, 0, st>>>(make_blocked(g, g.shape), U, mu.as<__half2>());
    note_launches(1);
    return run_inner_apply(g, W16<R1>{GaugeP16{mu.as<__half2>()}}, in, out, nsys, masses, r, dagger, st);
  }
  return SW_ERR_ARG;
}

int wilson_inner_apply(const Geom& g, const double2* U, const double2* in, double2* out, int nsys,
                       const double* masses, double r, int dagger, int precision, cudaStream_t st) {
  return (r == 1.0) ? inner_impl<true>(g, U, in, out, nsys, masses, r, dagger, precision, st)
                    : inner_impl<false>(g, U, in, out, nsys, masses, r, dagger, precision, st);
}

}  // namespace swc
