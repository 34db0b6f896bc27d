// Lambda(Omega, s*) of Section 3.2: the largest error of the local kernel
// approximation, sup over s in Omega of |k_approx(s, s*) - k(s, s*)| with
// k_approx(s, s*) = sum_q W_q k(s, s_q) over the 2L x 2L neighbours s_q of
// s* and K_N W = k(s*) (Eq. weights), for s* at the centre of the central
// box.  Omega is the plan's extent, the supremum is taken over a mesh of
// spacing (hx / sub, hy / sub) covering it.
//
// kerr_weights_kernel (one thread): K_N and k(s*) from the Matern
// correlation, K_N's Cholesky factor, two substitutions -> W (as the oracle
// does it).  kerr_sup_kernel: one thread per mesh point, the block's maximum
// in shared memory, then one atomic maximum on the double's bit pattern
// (non-negative doubles order like their bits).
#include "common.cuh"
#include "matern.cuh"

namespace rk {

__global__ void kerr_weights_kernel(int L, double hx, double hy, double rho, double sigma2,
                                    int nu_code, double* __restrict__ w, int* flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int MM = 64;
  const int W = 2 * L, M = W * W;
  double A[MM * (MM + 1) / 2];   // packed lower triangle, row i at i (i + 1) / 2
  double k[MM];
  // neighbour q = a + W b at ((a - (L - 1)) hx, (b - (L - 1)) hy) from the box
  // corner; s* at (hx / 2, hy / 2)
  for (int q = 0; q < M; ++q) {
    const int a = q % W, b = q / W;
    const double dx = (a - (L - 1) - 0.5) * hx, dy = (b - (L - 1) - 0.5) * hy;
    k[q] = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
    for (int r = 0; r <= q; ++r) {
      const int a2 = r % W, b2 = r / W;
      const double ex = (a - a2) * hx, ey = (b - b2) * hy;
      A[q * (q + 1) / 2 + r] = sigma2 * matern_phi<double>(sqrt(ex * ex + ey * ey) / rho, nu_code);
    }
  }
  for (int j = 0; j < M; ++j) {
    double d = A[j * (j + 1) / 2 + j];
    for (int t = 0; t < j; ++t) d -= A[j * (j + 1) / 2 + t] * A[j * (j + 1) / 2 + t];
    if (!(d > 0.0)) {
      *flag = 1;
      return;
    }
    d = sqrt(d);
    A[j * (j + 1) / 2 + j] = d;
    for (int i = j + 1; i < M; ++i) {
      double v = A[i * (i + 1) / 2 + j];
      for (int t = 0; t < j; ++t) v -= A[i * (i + 1) / 2 + t] * A[j * (j + 1) / 2 + t];
      A[i * (i + 1) / 2 + j] = v / d;
    }
  }
  for (int i = 0; i < M; ++i) {
    double v = k[i];
    for (int t = 0; t < i; ++t) v -= A[i * (i + 1) / 2 + t] * k[t];
    k[i] = v / A[i * (i + 1) / 2 + i];
  }
  for (int i = M - 1; i >= 0; --i) {
    double v = k[i];
    for (int t = i + 1; t < M; ++t) v -= A[t * (t + 1) / 2 + i] * k[t];
    k[i] = v / A[i * (i + 1) / 2 + i];
  }
  for (int q = 0; q < M; ++q) w[q] = k[q];
}

__global__ void __launch_bounds__(256)
kerr_sup_kernel(const double* __restrict__ w, int L, double x0, double y0, double hx,
                double hy, int i0, int j0, int sub, int mx, int my, double rho, double sigma2,
                int nu_code, unsigned long long* __restrict__ out) {
  const int W = 2 * L, M = W * W;
  __shared__ double ws[64];
  __shared__ double red[256];
  for (int q = threadIdx.x; q < M; q += blockDim.x) ws[q] = w[q];
  __syncthreads();
  const double sx = x0 + (i0 + 0.5) * hx, sy = y0 + (j0 + 0.5) * hy;
  double worst = 0.0;
  const long long total = (long long)mx * my;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(t % mx), iy = (int)(t / mx);
    const double px = x0 + ix * (hx / sub), py = y0 + iy * (hy / sub);
    double apx = 0.0;
    for (int q = 0; q < M; ++q) {
      const double nx = x0 + (i0 - (L - 1) + q % W) * hx, ny = y0 + (j0 - (L - 1) + q / W) * hy;
      const double dx = px - nx, dy = py - ny;
      apx = fma(ws[q], sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code), apx);
    }
    const double dx = px - sx, dy = py - sy;
    const double e = fabs(apx - sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code));
    worst = e > worst ? e : worst;
  }
  red[threadIdx.x] = worst;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s && red[threadIdx.x + s] > red[threadIdx.x])
      red[threadIdx.x] = red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

cudaError_t launch_kernel_error(const rk_plan* p, int sub, double* scratch, cudaStream_t s) {
  // scratch: M doubles of W, then the result's bits
  unsigned long long* res = reinterpret_cast<unsigned long long*>(scratch + 64);
  cudaError_t e = cudaMemsetAsync(res, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  kerr_weights_kernel<<<1, 32, 0, s>>>(p->L, p->hx, p->hy, p->rho, p->sigma2, p->nu_code,
                                       scratch, p->d_flag);
  const int i0 = (p->nx - 2) / 2, j0 = (p->ny - 2) / 2;
  const int mx = (p->nx - 1) * sub + 1, my = (p->ny - 1) * sub + 1;
  const long long total = (long long)mx * my;
  long long blocks = (total + 255) / 256;
  blocks = blocks > 4096 ? 4096 : blocks;
  kerr_sup_kernel<<<(unsigned)blocks, 256, 0, s>>>(scratch, p->L, p->x0, p->y0, p->hx, p->hy,
                                                   i0, j0, sub, mx, my, p->rho, p->sigma2,
                                                   p->nu_code, res);
  return cudaGetLastError();
}

}  // namespace rk
