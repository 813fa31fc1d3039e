// Scenario 4 (Sec. 2.1.4): the window functions of the partition of unity over the original
// CDD and the CDDs shifted by half a block, and the windowed input phi_ab r of the CDD
// shifted by (a, b) half blocks along (x, y).
//
// Along one axis of nb blocks of width s the unshifted interior cuts lie at k s (k = 1 ..
// nb - 1) and the shifted ones at s / 2 + k s (k = 0 .. nb - 1), in bulk node widths from
// the start of the bulk (node p's centre at p + 1/2).  A node at distance d_0 from the
// nearest unshifted cut and d_1 from the nearest shifted one has t = (d_0 - 1/2) /
// (d_0 + d_1 - 1) clipped to [0, 1] (t = 1 without unshifted cuts), psi_0 = sin^2(pi t / 2)
// and psi_1 = 1 - psi_0: psi_0 vanishes on the two node lines either side of every
// unshifted cut, psi_1 on those of every shifted cut, and phi_ab(x, y) = psi_a(x) psi_b(y)
// sums to one over the four CDDs.
#include <math.h>

#include "internal.h"

namespace lsw {

// psi[(axis * 2 + family) * Ne + P]: axis 0 = x (nb = r), 1 = y (nb = q)
__global__ void k_window_tables(double* __restrict__ psi, int Ne, int n, int npml, int nbx,
                                int nby) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * Ne) return;
  const int axis = t / Ne, P = t - axis * Ne;
  const int nb = axis == 0 ? nbx : nby;
  const int s = n / nb;
  const double x = (double)(P - npml) + 0.5;
  double tt = 1.0;
  if (nb > 1) {
    double d0 = INFINITY, d1 = INFINITY;
    for (int k = 1; k < nb; ++k) d0 = fmin(d0, fabs(x - (double)k * s));
    for (int k = 0; k < nb; ++k) d1 = fmin(d1, fabs(x - ((double)(s / 2) + (double)k * s)));
    tt = fmin(1.0, fmax(0.0, (d0 - 0.5) / (d0 + d1 - 1.0)));
  }
  const double sp = sinpi(0.5 * tt);
  const double p0 = sp * sp;
  psi[(axis * 2 + 0) * Ne + P] = p0;
  psi[(axis * 2 + 1) * Ne + P] = 1.0 - p0;
}

// out = phi_ab r on the extended grid (x fastest, then y, then z)
__global__ void k_window(const double2* __restrict__ r, double2* __restrict__ out,
                         const double* __restrict__ psi_x, const double* __restrict__ psi_y,
                         int Ne, long long N) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % Ne);
    const int y = (int)((e / Ne) % Ne);
    const double w = psi_x[x] * psi_y[y];
    const double2 v = r[e];
    out[e] = make_double2(w * v.x, w * v.y);
  }
}

cudaError_t launch_window_tables(Ctx& c) {
  const int th = 256, nb = (2 * c.Ne + th - 1) / th;
  k_window_tables<<<nb, th, 0, c.stream>>>(c.d_psi, c.Ne, c.n, c.npml, c.p.cdd_r, c.p.cdd_q);
  return cudaGetLastError();
}

cudaError_t launch_window(Ctx& c, const double2* r, double2* out, int a, int b) {
  const long long N = c.Next;
  const int th = 256;
  const long long nb = std::min<long long>((N + th - 1) / th, 152LL * 16);
  k_window<<<(unsigned)nb, th, 0, c.stream>>>(r, out, c.d_psi + (0 * 2 + a) * c.Ne,
                                               c.d_psi + (1 * 2 + b) * c.Ne, c.Ne, N);
  return cudaGetLastError();
}

}  // namespace lsw
