// Setup kernels: normal extension of m, PML tables and the coefficients of the global and
// local operators (Sec. 1.2, App. A; local problems of Sec. 2.2).
#include <math.h>

#include "internal.h"

namespace lsw {

// m_ext(P) = m_bulk(clamp(P - npml)) along every axis: constant extension along the
// normal of the bulk boundary (Sec. 1.2).
__global__ void k_extend_m(const double* __restrict__ mb, double* __restrict__ me, int n,
                           int npml, int Ne, int dim, long long Next) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= Next) return;
  int x = (int)(t % Ne);
  int y = (int)((t / Ne) % Ne);
  int z = dim == 3 ? (int)(t / ((long long)Ne * Ne)) : 0;
  int bx = min(max(x - npml, 0), n - 1);
  int by = min(max(y - npml, 0), n - 1);
  int bz = dim == 3 ? min(max(z - npml, 0), n - 1) : 0;
  me[t] = mb[((long long)bz * n + by) * n + bx];
}

cudaError_t launch_extend_m(Ctx& c, const double* m_bulk) {
  int th = 256;
  long long nb = (c.Next + th - 1) / th;
  k_extend_m<<<(unsigned)nb, th, 0, c.stream>>>(m_bulk, c.d_m_ext, c.n, c.npml, c.Ne, c.dim,
                                                c.Next);
  return cudaGetLastError();
}

// alpha_k = 1 / (1 + i sigma/omega) with the cubic profile of App. A measured from the
// interval [lo, hi] on which sigma vanishes; sigma = s (C/delta)(d/delta)^3 with s = omega
// (frequency-scaled reading) or s = 1 (literal).
__device__ double2 alpha_at(double x, double lo, double hi, double delta, double Cs,
                            double omega) {
  double d = 0.0;
  if (x < lo) d = lo - x;
  else if (x > hi) d = x - hi;
  double t = d / delta;
  double sigma = Cs / delta * t * t * t;
  // 1 / (1 + i sigma/omega)
  double a = sigma / omega;
  double den = 1.0 / (1.0 + a * a);
  return make_double2(den, -a * den);
}

__global__ void k_alpha_tables(const AlphaSeg* __restrict__ segs, int nseg, double2* tab,
                               double h, int npml, double delta, double Cs, double omega) {
  int s = blockIdx.y;
  if (s >= nseg) return;
  AlphaSeg g = segs[s];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * g.len + 1;
       t += gridDim.x * blockDim.x) {
    double x;
    if (t < g.len) x = (g.P0 + t - npml + 0.5) * h;      // node
    else x = (g.P0 + (t - g.len) - npml) * h;            // face below node (t - len)
    tab[g.off + t] = alpha_at(x, g.lo, g.hi, delta, Cs, omega);
  }
}

cudaError_t launch_alpha_tables(Ctx& c, const AlphaSeg* d_segs, int nseg, int max_len) {
  double delta = c.npml * c.h;
  double Cs = c.C * (c.p.pml_literal ? 1.0 : c.omega);
  dim3 grid((2 * max_len + 1 + 127) / 128, nseg);
  k_alpha_tables<<<grid, 128, 0, c.stream>>>(d_segs, nseg, c.d_alpha, c.h, c.npml, delta, Cs,
                                             c.omega);
  return cudaGetLastError();
}

// Coefficients of the symmetric operator on a box (Eq. Hemholtz_Symmetric, App. A):
//   d  = h^-2 sum_a (s_a(face below) + s_a(face above)) - omega^2 m / prod alpha
//   c_a = -h^-2 s_a(face above)  (coupling to the +1 neighbour along axis a; 0 on the
//   last node), s_a = alpha_a(face) / prod_{b != a} alpha_b(node).
template <typename CT>
__device__ void box_coeff(const SubGeom& g, int dim, const double2* __restrict__ tab,
                          const double* __restrict__ mext, int Ne, double omega, double ih2,
                          long long t, CT* out, long long stride) {
  int x = (int)(t % g.Lx);
  int y = (int)((t / g.Lx) % g.Ly);
  int z = (int)(t / ((long long)g.Lx * g.Ly));
  double2 one = make_double2(1.0, 0.0);
  double2 ax = tab[g.ax_tab + x], ay = tab[g.ay_tab + y];
  double2 az = dim == 3 ? tab[g.az_tab + z] : one;
  double2 fx0 = tab[g.ax_tab + g.Lx + x], fx1 = tab[g.ax_tab + g.Lx + x + 1];
  double2 fy0 = tab[g.ay_tab + g.Ly + y], fy1 = tab[g.ay_tab + g.Ly + y + 1];
  double2 fz0 = one, fz1 = one;
  if (dim == 3) { fz0 = tab[g.az_tab + g.Lz + z]; fz1 = tab[g.az_tab + g.Lz + z + 1]; }
  double2 ayz = cmul(ay, az), axz = cmul(ax, az), axy = cmul(ax, ay);
  double2 sx0 = cdiv(fx0, ayz), sx1 = cdiv(fx1, ayz);
  double2 sy0 = cdiv(fy0, axz), sy1 = cdiv(fy1, axz);
  double2 sum = sx0 + sx1 + sy0 + sy1;
  double2 sz1 = make_double2(0, 0);
  if (dim == 3) {
    double2 sz0 = cdiv(fz0, axy);
    sz1 = cdiv(fz1, axy);
    sum = sum + sz0 + sz1;
  }
  long long gi = ((long long)(g.gz0 + z) * Ne + (g.gy0 + y)) * Ne + (g.gx0 + x);
  double2 prod = dim == 3 ? cmul(axy, az) : axy;
  double2 mass = cdiv(make_double2(omega * omega * mext[gi], 0.0), prod);
  double2 d = make_double2(ih2 * sum.x - mass.x, ih2 * sum.y - mass.y);
  double2 cx = x < g.Lx - 1 ? make_double2(-ih2 * sx1.x, -ih2 * sx1.y) : make_double2(0, 0);
  double2 cy = y < g.Ly - 1 ? make_double2(-ih2 * sy1.x, -ih2 * sy1.y) : make_double2(0, 0);
  double2 cz = (dim == 3 && z < g.Lz - 1) ? make_double2(-ih2 * sz1.x, -ih2 * sz1.y)
                                          : make_double2(0, 0);
  long long o = g.node_off + t;
  out[o] = to<CT>(d);
  out[o + stride] = to<CT>(cx);
  out[o + 2 * stride] = to<CT>(cy);
  out[o + 3 * stride] = to<CT>(cz);
}

template <typename CT>
__global__ void k_local_coeff(const SubGeom* __restrict__ subs, int dim,
                              const double2* __restrict__ tab, const double* __restrict__ mext,
                              int Ne, double omega, double ih2, CT* out, long long stride) {
  SubGeom g = subs[blockIdx.y];
  long long nn = (long long)g.Lx * g.Ly * g.Lz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x)
    box_coeff<CT>(g, dim, tab, mext, Ne, omega, ih2, t, out, stride);
}

__global__ void k_global_coeff(SubGeom g, int dim, const double2* __restrict__ tab,
                               const double* __restrict__ mext, int Ne, double omega,
                               double ih2, double2* out, long long stride) {
  long long nn = (long long)g.Lx * g.Ly * g.Lz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x)
    box_coeff<double2>(g, dim, tab, mext, Ne, omega, ih2, t, out, stride);
}

cudaError_t launch_coefficients(Ctx& c) {
  double ih2 = 1.0 / (c.h * c.h);
  SubGeom g{};
  g.Lx = c.Ne; g.Ly = c.Ne; g.Lz = c.dim == 3 ? c.Ne : 1;
  g.ax_tab = g.ay_tab = g.az_tab = c.alpha_global_tab;
  g.node_off = 0;
  long long nb = (c.Next + 255) / 256;
  if (nb > 65535LL * 8) nb = 65535LL * 8;
  k_global_coeff<<<(unsigned)nb, 256, 0, c.stream>>>(g, c.dim, c.d_alpha, c.d_m_ext, c.Ne,
                                                     c.omega, ih2, c.d_gcoef, c.Next);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long per = 0;
  for (auto& s : c.subs) per = std::max(per, (long long)s.Lx * s.Ly * s.Lz);
  dim3 grid((unsigned)std::min<long long>((per + 255) / 256, 4096), (unsigned)c.subs.size());
  if (c.c64())
    k_local_coeff<float2><<<grid, 256, 0, c.stream>>>(c.d_subs, c.dim, c.d_alpha, c.d_m_ext,
                                                      c.Ne, c.omega, ih2, (float2*)c.d_lcoef,
                                                      c.node_elems);
  else
    k_local_coeff<double2><<<grid, 256, 0, c.stream>>>(c.d_subs, c.dim, c.d_alpha, c.d_m_ext,
                                                       c.Ne, c.omega, ih2, (double2*)c.d_lcoef,
                                                       c.node_elems);
  return cudaGetLastError();
}

// f_ext = f on the bulk, 0 in the PML (f / prod alpha = f there since alpha = 1).
__global__ void k_extend_source(const double* __restrict__ fb, double2* __restrict__ fe, int n,
                                int npml, int Ne, int dim, long long Next) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= Next) return;
  int x = (int)(t % Ne) - npml;
  int y = (int)((t / Ne) % Ne) - npml;
  int z = dim == 3 ? (int)(t / ((long long)Ne * Ne)) - npml : 0;
  bool in = x >= 0 && x < n && y >= 0 && y < n && z >= 0 && z < n;
  fe[t] = make_double2(in ? fb[((long long)z * n + y) * n + x] : 0.0, 0.0);
}

cudaError_t launch_extend_source(Ctx& c, const double* f_bulk, double2* f_ext) {
  long long nb = (c.Next + 255) / 256;
  k_extend_source<<<(unsigned)nb, 256, 0, c.stream>>>(f_bulk, f_ext, c.n, c.npml, c.Ne, c.dim,
                                                      c.Next);
  return cudaGetLastError();
}

}  // namespace lsw
