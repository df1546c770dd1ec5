// sft_noalloc.cu -- flux diagnostics of one caller-owned device map with no
// device allocation at all.
//
// Who needs this: code that cannot call cudaMalloc once it is running, for
// example a solver coupled into a larger model that has already reserved
// nearly all device memory through its own pool (an allocation would fail,
// or force the pool to release and fragment memory), or a real-time
// pipeline that forbids allocation after start-up because cudaMalloc can
// synchronise the device and stall it.  Such callers hold their map in
// memory they own and only need the analysis quantities.
//
// All scratch (the map descriptor, the row/column tables, the per-block
// partial sums and the folded result) lives in one file-scope __device__
// array of SFT_NOALLOC_SCRATCH_BYTES.  Every GPU that loads libsft holds that
// array until the process exits.  Host code cannot use the array's name as
// a device address (in host code it names a host-side stand-in), so every
// call asks the runtime for the array's address in the current context with
// cudaGetSymbolAddress (a lookup that allocates nothing), which stays right
// after a cudaDeviceReset or inside a caller's own driver-API context.
// With lazy module loading (CUDA's default) the first call in a context is
// also the moment the runtime loads this library's device code and commits
// the array's memory: a caller whose memory pool takes the device must make
// one call at start-up, before the pool reserves its memory, or load the
// library with CUDA_MODULE_LOADING=EAGER.  Every call shares the one array
// and overwrites all of it that it reads (nothing needs to start at zero),
// so calls whose work overlaps on the GPU race: serialise them (one stream,
// or synchronise between calls).  A call returns only after its result has
// reached the host: it waits for cuda_stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "sft.h"
#include "sft_device.cuh"

namespace sft {
void set_global_error(const std::string& msg);  // sft_api.cu (sft_last_error(NULL))
}

using namespace sft;

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[SFT_NOALLOC_SCRATCH_BYTES];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t desc, tiles, start, geod, cosp, sinp, csf, partials, out, total;
  int n_tiles, band;
};

Layout layout(int nt, int np) {
  Layout L{};
  L.band = np >= 32768 ? 1 : 32768 / np;
  L.n_tiles = (nt + L.band - 1) / L.band;
  size_t o = 0;
  L.desc = o;     o = align256(o + sizeof(RealDesc));
  L.tiles = o;    o = align256(o + (size_t)L.n_tiles * sizeof(RedTile));
  L.start = o;    o = align256(o + 2 * sizeof(int));
  L.geod = o;     o = align256(o + (size_t)nt * sizeof(RowGeoD));
  L.cosp = o;     o = align256(o + (size_t)np * sizeof(double));
  L.sinp = o;     o = align256(o + (size_t)np * sizeof(double));
  L.csf = o;      o = align256(o + (size_t)np * sizeof(float4));
  L.partials = o; o = align256(o + (size_t)L.n_tiles * kDiagFields * sizeof(double));
  L.out = o;      o = align256(o + kDiagFields * sizeof(double));
  L.total = o;
  return L;
}

// Fill the descriptor and the geometry tables of an nt x np map (pitch np)
// inside the scratch: the same quantities sft_create_grid tabulates on the
// host (Sec. 3.2 grid, App. A cap area), computed here in FP64 on the device.
__global__ void noalloc_tables_kernel(unsigned char* base, Layout L, int nt, int np) {
  const double pi = 3.14159265358979323846;
  const double dth = pi / (nt - 1), dph = 2.0 * pi / np;
  const double cap = 2.0 * pi * (1.0 - cos(0.5 * dth));
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  if (tid == 0) {
    RealDesc d{};
    d.nt = nt;
    d.np = np;
    d.pitch = np;
    *reinterpret_cast<RealDesc*>(base + L.desc) = d;
    int* st = reinterpret_cast<int*>(base + L.start);
    st[0] = 0;
    st[1] = L.n_tiles;
  }
  RedTile* tl = reinterpret_cast<RedTile*>(base + L.tiles);
  for (int t = tid; t < L.n_tiles; t += nth) {
    const int j0 = t * L.band;
    tl[t] = RedTile{0, j0, min(nt, j0 + L.band), 0};
  }
  RowGeoD* gd = reinterpret_cast<RowGeoD*>(base + L.geod);
  for (int j = tid; j < nt; j += nth) {
    const bool pole = j == 0 || j == nt - 1;
    const double th = j == nt - 1 ? pi : j * dth;
    RowGeoD g;
    g.sin_t = pole ? 0.0 : sin(th);
    g.cos_t = cos(th);
    g.lat = 0.5 * pi - th;
    g.area = pole ? cap / np : g.sin_t * dth * dph;
    gd[j] = g;
  }
  double* cp = reinterpret_cast<double*>(base + L.cosp);
  double* sp = reinterpret_cast<double*>(base + L.sinp);
  float4* cf = reinterpret_cast<float4*>(base + L.csf);
  for (int k = tid; k < np; k += nth) {
    const double c = cos(k * dph), s = sin(k * dph);
    cp[k] = c;
    sp[k] = s;
    const float ch = (float)c, sh = (float)s;
    cf[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
}

sft_status noalloc_fail(sft_status code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

}  // namespace

extern "C" sft_status sft_flux_diagnostics_noalloc(const void* br_device, int32_t ntheta, int32_t nphi,
                                                   sft_prec prec, double lat_cut_deg,
                                                   void* cuda_stream, sft_diag* out) {
  if (!br_device || !out) return noalloc_fail(SFT_ERR_ARG, "noalloc diagnostics: NULL argument");
  if (prec != SFT_FP32 && prec != SFT_FP64) return noalloc_fail(SFT_ERR_ARG, "noalloc diagnostics: bad precision");
  if (ntheta < 5 || nphi < 8 || ntheta > (1 << 20) || nphi > (1 << 20))
    return noalloc_fail(SFT_ERR_ARG, "noalloc diagnostics: shape out of range (ntheta >= 5, nphi >= 8)");
  const Layout L = layout(ntheta, nphi);
  if (L.total > SFT_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(SFT_ERR_ARG, "noalloc diagnostics: a " + std::to_string(ntheta) + "x" +
                                         std::to_string(nphi) + " map needs " + std::to_string(L.total) +
                                         " bytes of scratch, more than the fixed " +
                                         std::to_string((size_t)SFT_NOALLOC_SCRATCH_BYTES) + "-byte array");
  // The array's device address in the current context (looked up on every
  // call, never cached: a cached address goes stale when the context does).
  void* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess)
    return noalloc_fail(SFT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  noalloc_tables_kernel<<<std::max(1, std::min(1024, (std::max(ntheta, nphi) + 255) / 256)), 256, 0, st>>>(
      b, L, ntheta, nphi);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(SFT_ERR_CUDA, std::string("tables kernel: ") + cudaGetErrorString(e));
  const auto* desc = reinterpret_cast<const RealDesc*>(b + L.desc);
  const auto* tiles = reinterpret_cast<const RedTile*>(b + L.tiles);
  const auto* geod = reinterpret_cast<const RowGeoD*>(b + L.geod);
  const auto* cosp = reinterpret_cast<const double*>(b + L.cosp);
  const auto* sinp = reinterpret_cast<const double*>(b + L.sinp);
  const auto* csf = reinterpret_cast<const float4*>(b + L.csf);
  auto* partials = reinterpret_cast<double*>(b + L.partials);
  auto* res = reinterpret_cast<double*>(b + L.out);
  const double cut = lat_cut_deg * 3.14159265358979323846 / 180.0;
  AssimArgs aa{nullptr, nullptr, nullptr, nullptr};
  e = prec == SFT_FP32
          ? launch_reduce<float>(RED_DIAG, L.n_tiles, st, tiles, desc, geod, cosp, sinp, csf,
                                 static_cast<const float*>(br_device), cut, aa, partials)
          : launch_reduce<double>(RED_DIAG, L.n_tiles, st, tiles, desc, geod, cosp, sinp, csf,
                                  static_cast<const double*>(br_device), cut, aa, partials);
  if (e != cudaSuccess) return noalloc_fail(SFT_ERR_CUDA, std::string("reduce: ") + cudaGetErrorString(e));
  e = launch_fold(RED_DIAG, 1, st, reinterpret_cast<const int*>(b + L.start), partials, nullptr, res);
  if (e != cudaSuccess) return noalloc_fail(SFT_ERR_CUDA, std::string("fold: ") + cudaGetErrorString(e));
  double v[kDiagFields];
  e = cudaMemcpyAsync(v, res, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(SFT_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
  const double mx = 6.96e10 * 6.96e10;  // R_sun^2 in cm^2 (Sec. 3.3)
  const double k3 = 3.0 / (4.0 * 3.14159265358979323846);
  out->flux_signed = v[0] * mx;
  out->flux_pos = v[1] * mx;
  out->flux_neg = v[2] * mx;
  out->flux_pole_n = v[3] * mx;
  out->flux_pole_s = v[4] * mx;
  out->area_pole_n = v[5] * mx;
  out->area_pole_s = v[6] * mx;
  out->dipole_axial = k3 * v[7];
  out->h1 = k3 * v[8];
  out->h2 = k3 * v[9];
  out->nonfinite = (int64_t)v[10];
  out->brmin = v[11];
  out->brmax = v[12];
  out->absmin = v[13];
  out->t_hours = 0.0;
  out->steps = 0;
  return SFT_OK;
}
