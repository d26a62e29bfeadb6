// Pieces of the DMK far field shared by the 3D (far.cu) and 2D (far2d.cu) paths:
// element types, the barycentric Lagrange row at the Chebyshev points of the
// first kind, the window transform gamma-hat and the Table 2 proxy order.
#pragma once
#include "common.cuh"
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace dmk {
namespace farc {

constexpr int kMaxP = 64;          // proxy order and mode counts a side (Table 2 needs <= 63)

struct BoxGeo {
  double x, y, z, w;   // centre and half side, in-cell coordinates
};

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// four consecutive entries from 16-byte aligned shared memory
__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const float2* p, float2* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 2);
  v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void ld4(const double2* p, double2* v) {
  v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
}

// 1 / d in the far field's precision: the correctly rounded reciprocal in float32
// (one reciprocal per node serves the barycentric sum and the values), a division in
// float64
template <typename R> __device__ __forceinline__ R recip(R d);
template <> __device__ __forceinline__ float recip<float>(float d) { return __frcp_rn(d); }
template <> __device__ __forceinline__ double recip<double>(double d) { return 1.0 / d; }

// Lagrange basis at the Chebyshev points of the first kind in barycentric form
// (weights (-1)^j sin((2j+1) pi / 2p)), in the far field's precision:
// L_j(t) = (w_j / (t - x_j)) / sum_k w_k / (t - x_k), exact at a node;
// out[j * stride] for j < pad (zero past p)
template <typename R>
__device__ inline void lagrange_row(R t, int p, const R* nodes, const R* bw, R* out, int stride, int pad) {
  R s = R(0);
  int hit = -1;
  for (int j = 0; j < p; ++j) {
    const R d = t - nodes[j];
    R v = R(0);
    if (d == R(0)) hit = j;
    else v = bw[j] * recip<R>(d);
    out[j * stride] = v;
    s += v;
  }
  const R inv = hit >= 0 ? R(0) : recip<R>(s);
  for (int j = 0; j < pad; ++j) {
    R v = R(0);
    if (j < p) v = hit >= 0 ? (j == hit ? R(1) : R(0)) : out[j * stride] * inv;
    out[j * stride] = v;
  }
}

// gamma-hat(kappa) = 2 int_0^1 phi(t) (cos(kappa t) + kappa t sin(kappa t) / 2) dt
// (Eq. (gammaB_in_phi)), Gauss-Legendre on [0, 1]
struct GammaHat {
  std::vector<double> t, wphi;
  explicit GammaHat(double c) {
    ProlateSeries ser;
    if (prolate_series(c, &ser) != 0) throw Error{DMK_ERR_CUDA, "prolate series failed"};
    std::vector<double> x, w;
    gauss_legendre(256, x, w);
    t.resize(x.size());
    wphi.resize(x.size());
    for (size_t i = 0; i < x.size(); ++i) {
      t[i] = 0.5 * (x[i] + 1.0);
      wphi[i] = w[i] * series_phi(ser, t[i]);       // 2 * (1/2) w_i phi(t_i)
    }
  }
  double operator()(double kap) const {
    double s = 0.0;
    for (size_t i = 0; i < t.size(); ++i) s += wphi[i] * (std::cos(kap * t[i]) + 0.5 * kap * t[i] * std::sin(kap * t[i]));
    return s;
  }
};

// Table 2 columns and the rules that reproduce them: N1 = 2 (3c/pi) - 1, N_per = 2 floor(c / 2pi) + 1;
// p interpolated linearly in log10 eps between the rows and rounded up
inline int table2_p(double eps, int kernels) {
  static const double e_rows[4] = {-12, -9, -6, -3};
  static const double p_s[4] = {44, 33, 23, 12}, p_t[4] = {44, 33, 22, 11};
  const double e = std::log10(eps);
  auto interp = [&](const double* v) {
    for (int i = 0; i < 3; ++i)
      if (e >= e_rows[i] - 1e-9 && e <= e_rows[i + 1] + 1e-9) {
        const double tt = (e - e_rows[i]) / (e_rows[i + 1] - e_rows[i]);
        return static_cast<int>(std::ceil(v[i] + tt * (v[i + 1] - v[i]) - 1e-9));
      }
    return static_cast<int>(v[0]);
  };
  int p = 0;
  if (kernels & DMK_KERNEL_STOKESLET) p = std::max(p, interp(p_s));
  if (kernels & DMK_KERNEL_STRESSLET) p = std::max(p, interp(p_t));
  return p;
}

namespace {
// copies segment b of the packed upload: desc[b] = (source word offset, word count,
// destination address as two 32-bit halves)
__global__ void k_scatter_words(const uint32_t* __restrict__ packed, const int4* __restrict__ desc) {
  const int4 d = desc[blockIdx.x];
  uint32_t* dst = reinterpret_cast<uint32_t*>((static_cast<uint64_t>(static_cast<uint32_t>(d.w)) << 32) |
                                              static_cast<uint32_t>(d.z));
  const uint32_t* src = packed + d.x;
  for (int i = threadIdx.x; i < d.y; i += blockDim.x) dst[i] = src[i];
}
}  // namespace

// the plan's small device tables: put() takes each table's device place from the
// plan's arena at once and keeps a packed host copy; flush() moves them all with one
// host-to-device copy and one scatter launch (instead of one copy per table)
struct Uploader {
  Plan& p;
  std::vector<uint32_t> packed;         // host words of every table, each 16-byte aligned
  std::vector<int4> desc;
  explicit Uploader(Plan& plan) : p(plan) {}
  template <typename T>
  T* put(const std::vector<T>& v) {
    if ((v.size() * sizeof(T)) % 4) throw Error{DMK_ERR_CUDA, "device table not a whole number of words"};
    T* d = p.arena.alloc<T>(std::max<size_t>(v.size(), 1));
    if (v.empty()) return d;
    const size_t off = (packed.size() + 3) & ~size_t(3);
    const size_t words = v.size() * sizeof(T) / 4;
    packed.resize(off + words);
    std::memcpy(packed.data() + off, v.data(), v.size() * sizeof(T));
    const uint64_t a = reinterpret_cast<uint64_t>(d);
    desc.push_back(make_int4(static_cast<int>(off), static_cast<int>(words), static_cast<int>(a & 0xffffffffu),
                             static_cast<int>(a >> 32)));
    return d;
  }
  void flush() {
    if (desc.empty()) return;
    const size_t doff = (packed.size() + 3) & ~size_t(3);
    packed.resize(doff + desc.size() * 4);
    std::memcpy(packed.data() + doff, desc.data(), desc.size() * sizeof(int4));
    uint32_t* d = p.arena.alloc<uint32_t>(packed.size());
    DMK_CUDA_TRY(cudaMemcpyAsync(d, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice, p.stream));
    k_scatter_words<<<static_cast<unsigned>(desc.size()), 256, 0, p.stream>>>(d, reinterpret_cast<const int4*>(d + doff));
    DMK_CUDA_TRY(cudaGetLastError());
    ++p.launches;
    packed.clear();
    desc.clear();
  }
};

// incoming expansions, phase e^{-2 pi i m.delta / 3} for a colleague at offset delta
// (e = m.delta mod 3: 1, e^{-2 pi i/3}, e^{-4 pi i/3})
template <typename R>
__device__ __forceinline__ void add_phased(int e, R ox, R oy, R& sr, R& si) {
  const R c120 = R(-0.5), s120 = R(0.86602540378443864676);
  if (e == 0) {
    sr += ox;
    si += oy;
  } else {
    const R sn = e == 1 ? -s120 : s120;
    sr += c120 * ox - sn * oy;
    si += c120 * oy + sn * ox;
  }
}

// the phase e^{-2 pi i m.delta/3} factors over the axes: f(+1) = e^{-2 pi i m / 3} for
// a colleague one box further along an axis (mode m on that axis), f(-1) = conj f(+1)
template <typename R>
__device__ __forceinline__ void axis_phase(int m, R& c, R& s) {
  int e = m % 3;
  if (e < 0) e += 3;
  c = e == 0 ? R(1) : R(-0.5);
  s = e == 0 ? R(0) : (e == 1 ? R(-0.86602540378443864676) : R(0.86602540378443864676));
}
template <typename R>
__device__ __forceinline__ void sum3(R c, R s, R xr_m, R xi_m, R xr_0, R xi_0, R xr_p, R xi_p, R& yr, R& yi) {
  // y = f(-1) x_{-1} + x_0 + f(+1) x_{+1},  f(+1) = c + i s, f(-1) = c - i s
  yr = xr_0 + c * (xr_m + xr_p) + s * (xi_m - xi_p);
  yi = xi_0 + c * (xi_m + xi_p) + s * (xr_p - xr_m);
}

// ---- host: the parameter-only matrices ------------------------------------------
// Chebyshev points of the first kind cos((2j+1) pi / 2p) and their barycentric
// weights (-1)^j sin((2j+1) pi / 2p)
inline void cheb_nodes_bw(int P, std::vector<double>& nodes, std::vector<double>& bw) {
  nodes.resize(P);
  bw.resize(P);
  for (int j = 0; j < P; ++j) {
    const double th = (2.0 * j + 1.0) * M_PI / (2.0 * P);
    nodes[j] = std::cos(th);
    bw[j] = ((j & 1) ? -1.0 : 1.0) * std::sin(th);
  }
}

// L_j(t) as the plain Lagrange product over the nodes
inline double lagrange_host(const std::vector<double>& nodes, double t, int j) {
  double v = 1.0;
  for (size_t k = 0; k < nodes.size(); ++k)
    if (static_cast<int>(k) != j) v *= (t - nodes[k]) / (nodes[j] - nodes[k]);
  return v;
}

// a byte bank of real and complex matrices in the far field's precision, each
// entry 16-byte aligned; put_* return the entry's byte offset
struct MatBank {
  std::vector<char> bytes;
  bool f32 = true;
  size_t put_real(const std::vector<double>& v) {
    const size_t off = (bytes.size() + 15) & ~size_t(15);
    bytes.resize(off + v.size() * (f32 ? 4 : 8));
    for (size_t i = 0; i < v.size(); ++i) {
      if (f32) reinterpret_cast<float*>(bytes.data() + off)[i] = static_cast<float>(v[i]);
      else reinterpret_cast<double*>(bytes.data() + off)[i] = v[i];
    }
    return off;
  }
  size_t put_cplx(const std::vector<double>& re, const std::vector<double>& im) {
    const size_t off = (bytes.size() + 15) & ~size_t(15);
    bytes.resize(off + re.size() * (f32 ? 8 : 16));
    for (size_t i = 0; i < re.size(); ++i) {
      if (f32) {
        reinterpret_cast<float*>(bytes.data() + off)[2 * i] = static_cast<float>(re[i]);
        reinterpret_cast<float*>(bytes.data() + off)[2 * i + 1] = static_cast<float>(im[i]);
      } else {
        reinterpret_cast<double*>(bytes.data() + off)[2 * i] = re[i];
        reinterpret_cast<double*>(bytes.data() + off)[2 * i + 1] = im[i];
      }
    }
    return off;
  }
  // plane-wave matrix over modes m = lo .. lo + n - 1 at the nodes xi_j:
  //   outgoing (eval = false): E[m][j] = e^{-i theta m xi_j};
  //   evaluation (eval = true): F[j][m] = w_m e^{+i theta m xi_j}, w_m = 2 for m > 0
  //   when only the m >= 0 half of the axis is kept (half), else 1
  size_t plane_wave(const std::vector<double>& nodes, int lo, int n, double theta, bool eval, bool half) {
    const int P = static_cast<int>(nodes.size());
    std::vector<double> re(static_cast<size_t>(n) * P), im(re.size());
    for (int mi = 0; mi < n; ++mi)
      for (int j = 0; j < P; ++j) {
        const int m = lo + mi;
        const double ph = theta * m * nodes[j];
        const double wgt = (eval && half && m > 0) ? 2.0 : 1.0;
        const size_t e = eval ? static_cast<size_t>(j) * n + mi : static_cast<size_t>(mi) * P + j;
        re[e] = wgt * std::cos(ph);
        im[e] = (eval ? 1.0 : -1.0) * wgt * std::sin(ph);
      }
    return put_cplx(re, im);
  }
};

}  // namespace farc
}  // namespace dmk
