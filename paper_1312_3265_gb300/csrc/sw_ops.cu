// Staggered Wilson operator: FP64 apply (C ABI) and batched CGNE.
#include "driver.cuh"

namespace swc {

using SW64 = SWOp<double, GaugeC64, TransC64, VecC64>;
using SW32 = SWOp<float, GaugeP32, TransP32, VecP32x2>;
using SW16 = SWOp<float, GaugeP16, TransP16, VecP16>;

int sw_apply_f64(const Geom& g, const double2* U, const double2* W, const double2* in, double2* out,
                 double mass, double r, int dagger, cudaStream_t st) {
  const SW64 op{GaugeC64{U}, TransC64{W}};
  const int gx = (g.V + 127) / 128;
  apply_kernel<double, SW64><<<dim3(gx, 1), 128, 0, st>>>(g, op, VecC64<3>{const_cast<double2*>(in)},
                                                          VecC64<3>{out}, mass, 0, r, dagger,
                                                          nullptr, 0);
  note_launches(1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SW_OK : cuda_fail(e);
}

int sw_cgne(const Geom& g, const SolveArgs& a) {
  const SW64 opd{GaugeC64{a.U}, TransC64{a.W}};
  if (a.precision == SW_PREC_F64) return run_cgne<SW64, SW64, false>(g, opd, opd, a);
  if (a.precision == SW_PREC_F32_RELIABLE) {
    DevMem mu, mw;
    if (!mu.alloc(sizeof(float2) * 36 * (size_t)g.V, a.stream) ||
        !mw.alloc(sizeof(float2) * 72 * (size_t)g.V, a.stream))
      return SW_ERR_OOM;
    const int gp = sm_count() * 8;
    pack_mats_p32<<<gp, 256, 0, a.stream>>>(make_blocked(g, g.shape), 4, a.U, mu.as<float2>());
    pack_mats_p32<<<gp, 256, 0, a.stream>>>(make_blocked(g, g.shape), 8, a.W, mw.as<float2>());
    note_launches(2);
    const SW32 opf{GaugeP32{mu.as<float2>()}, TransP32{mw.as<float2>()}};
    return run_cgne<SW64, SW32, true>(g, opd, opf, a);
  }
  if (a.precision == SW_PREC_F16_RELIABLE) {
    if (int e = check_su3(g, a.U, a.stream)) return e;
    DevMem mu, mw;
    if (!mu.alloc(sizeof(__half2) * 24 * (size_t)g.V, a.stream) ||
        !mw.alloc(sizeof(__half2) * 72 * (size_t)g.V, a.stream))
      return SW_ERR_OOM;
    const int gp = sm_count() * 8;
    pack_links_h12<<<gp, 256, 0, a.stream>>>(make_blocked(g, g.shape), a.U, mu.as<__half2>());
    pack_mats_h<<<gp, 256, 0, a.stream>>>(make_blocked(g, g.shape), 8, a.W, mw.as<__half2>());
    note_launches(2);
    const SW16 opf{GaugeP16{mu.as<__half2>()}, TransP16{mw.as<__half2>()}};
    return run_cgne<SW64, SW16, true>(g, opd, opf, a);
  }
  return SW_ERR_ARG;
}


int sw_inner_apply(const Geom& g, const double2* U, const double2* W, const double2* in, double2* out, int nsys,
                   const double* masses, double r, int dagger, int precision, cudaStream_t st) {
  const int gp = sm_count() * 8;
  if (precision == SW_PREC_F32_RELIABLE) {
    DevMem mu, mw;
    if (!mu.alloc(sizeof(float2) * 36 * (size_t)g.V, st) || !mw.alloc(sizeof(float2) * 72 * (size_t)g.V, st))
      return SW_ERR_OOM;
    pack_mats_p32<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 4, U, mu.as<float2>());
    pack_mats_p32<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 8, W, mw.as<float2>());
    note_launches(2);
    return run_inner_apply(g, SW32{GaugeP32{mu.as<float2>()}, TransP32{mw.as<float2>()}}, in, out, nsys, masses, r,
                           dagger, st);
  }
  if (precision == SW_PREC_F16_RELIABLE) {
    if (int e = check_su3(g, U, st)) return e;
    DevMem mu, mw;
    if (!mu.alloc(sizeof(__half2) * 24 * (size_t)g.V, st) || !mw.alloc(sizeof(__half2) * 72 * (size_t)g.V, st))
      return SW_ERR_OOM;
    pack_links_h12<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), U, mu.as<__half2>());
    pack_mats_h<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 8, W, mw.as<__half2>());
    note_launches(2);
    return run_inner_apply(g, SW16{GaugeP16{mu.as<__half2>()}, TransP16{mw.as<__half2>()}}, in, out, nsys, masses,
                           r, dagger, st);
  }
  return SW_ERR_ARG;
}

}  // namespace swc
