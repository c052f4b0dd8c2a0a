// fft.cu -- hand-written 3D real FFT for the PM Poisson solve (paper Sec. 2.1:
// "combined in Fourier space using an exponential kernel") and for the
// initial conditions.
//
// Layout: real mesh [ix][iy][iz] (iz fastest), half spectrum [ix][iy][kz],
// kz in [0, n/2].  Five passes, each one read and one write of the mesh:
//   Z r2c  -- two real rows packed as one complex row, n-point FFT, unpacked;
//   Y      -- W spectrum columns (consecutive kz) per block, FFT along iy;
//   X      -- same along ix; for the Poisson solve the forward FFT, the Green
//             multiply and the inverse FFT are fused in one pass;
//   Y inverse, Z c2r.
// In-block transform: radix-2 decimation in time on shared memory, columns
// interleaved (element e of column q at e * W + q), bit-reversed load.
// Twiddles come from an FP64 host table (cast to the working precision).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dzs {
namespace {

constexpr int kFftThreads = 256;
constexpr int kSmemBytes = 64 * 1024;

template <class R>
__device__ void fft_smem(cplx<R>* buf, int n, int logn, int W, const cplx<R>* __restrict__ tw, bool inverse) {
  const int nb = (n >> 1) * W;
  for (int s = 0; s < logn; ++s) {
    const int half = 1 << s;
    const int stride = n >> (s + 1);  // twiddle index stride
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
      int col = q % W, b = q / W;
      int j = b & (half - 1);
      int i0 = ((b >> s) << (s + 1)) + j;
      int i1 = i0 + half;
      cplx<R> w = tw[j * stride];
      if (inverse) w.y = -w.y;
      cplx<R> a = buf[i0 * W + col];
      cplx<R> bb = cmul(buf[i1 * W + col], w);
      buf[i0 * W + col] = {a.x + bb.x, a.y + bb.y};
      buf[i1 * W + col] = {a.x - bb.x, a.y - bb.y};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int e, int logn) { return (int)(__brev((unsigned)e) >> (32 - logn)); }

// Z pass, real -> half spectrum.  Block handles W row pairs.
template <class R>
__global__ void k_fft_z_r2c(const R* __restrict__ in, cplx<R>* __restrict__ out, int n, int logn, int W,
                            int64_t npairs, const cplx<R>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw);
  const int64_t p0 = (int64_t)blockIdx.x * W;
  const int hn = n / 2 + 1;
  for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
    int col = q / n, e = q % n;
    int64_t pr = p0 + col;
    cplx<R> v = {0, 0};
    if (pr < npairs) v = {in[(2 * pr) * n + e], in[(2 * pr + 1) * n + e]};
    buf[bitrev(e, logn) * W + col] = v;
  }
  __syncthreads();
  fft_smem(buf, n, logn, W, tw, false);
  for (int q = threadIdx.x; q < hn * W; q += blockDim.x) {
    int col = q / hn, k = q % hn;
    int64_t pr = p0 + col;
    if (pr >= npairs) continue;
    cplx<R> z = buf[(k % n) * W + col], zc = buf[((n - k) % n) * W + col];
    // X_a = (Z_k + conj Z_-k) / 2,  X_b = (Z_k - conj Z_-k) / (2 i)
    cplx<R> xa = {(R)0.5 * (z.x + zc.x), (R)0.5 * (z.y - zc.y)};
    cplx<R> xb = {(R)0.5 * (z.y + zc.y), (R)-0.5 * (z.x - zc.x)};
    out[(2 * pr) * hn + k] = xa;
    out[(2 * pr + 1) * hn + k] = xb;
  }
}

// Z pass inverse, half spectrum -> real (unnormalised).  Block: W row pairs.
template <class R>
__global__ void k_fft_z_c2r(const cplx<R>* __restrict__ in, R* __restrict__ out, int n, int logn, int W,
                            int64_t npairs, const cplx<R>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw);
  const int64_t p0 = (int64_t)blockIdx.x * W;
  const int hn = n / 2 + 1;
  for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
    int col = q / n, k = q % n;
    int64_t pr = p0 + col;
    cplx<R> z = {0, 0};
    if (pr < npairs) {
      cplx<R> a, b;
      if (k < hn) {
        a = in[(2 * pr) * hn + k];
        b = in[(2 * pr + 1) * hn + k];
      } else {
        a = in[(2 * pr) * hn + (n - k)];
        b = in[(2 * pr + 1) * hn + (n - k)];
        a.y = -a.y;
        b.y = -b.y;
      }
      z = {a.x - b.y, a.y + b.x};  // a + i b
    }
    buf[bitrev(k, logn) * W + col] = z;
  }
  __syncthreads();
  fft_smem(buf, n, logn, W, tw, true);
  for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
    int col = q / n, e = q % n;
    int64_t pr = p0 + col;
    if (pr >= npairs) continue;
    cplx<R> z = buf[e * W + col];
    out[(2 * pr) * n + e] = z.x;
    out[(2 * pr + 1) * n + e] = z.y;
  }
}

// Column pass along Y (axis = 1) or X (axis = 0) of the half spectrum.
// mode 0 forward, 1 inverse, 2 forward + Green multiply + inverse (X only).
template <class R>
__global__ void k_fft_cols(cplx<R>* __restrict__ spec, int n, int logn, int W, int axis, int mode,
                           const cplx<R>* __restrict__ tw, const R* __restrict__ gtab, R gfac) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw);
  const int hn = n / 2 + 1;
  const int ncb = (hn + W - 1) / W;            // column blocks per line
  const int line = blockIdx.x / ncb;           // fixed other index (ix for Y, iy for X)
  const int kz0 = (blockIdx.x % ncb) * W;
  const int64_t es = axis == 1 ? (int64_t)hn : (int64_t)n * hn;     // element stride
  const int64_t base = axis == 1 ? (int64_t)line * n * hn : (int64_t)line * hn;
  for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
    int e = q / W, col = q % W;
    cplx<R> v = {0, 0};
    if (kz0 + col < hn) v = spec[base + e * es + kz0 + col];
    buf[bitrev(e, logn) * W + col] = v;
  }
  __syncthreads();
  fft_smem(buf, n, logn, W, tw, mode == 1);
  if (mode == 2) {
    // Green function: gtab holds per-axis k^2 (first n) and W_CIC^2 (next n)
    const R* k2t = gtab;
    const R* wt = gtab + n;
    for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
      int e = q / W, col = q % W;  // e = kx index
      int kz = kz0 + col;
      R gv = 0;
      if (kz < hn) {
        R k2 = k2t[e] + k2t[line] + k2t[kz];
        if (k2 > (R)0) {
          R w = wt[e] * wt[line] * wt[kz];
          gv = gfac * exp(-k2 * gtab[2 * n]) / (k2 * w * w);
        }
      }
      cplx<R> v = buf[e * W + col];
      buf[e * W + col] = {v.x * gv, v.y * gv};
    }
    __syncthreads();
    // bit-reverse in place for the inverse transform
    for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
      int e = q / W, col = q % W;
      int r = bitrev(e, logn);
      if (r > e) {
        cplx<R> t = buf[e * W + col];
        buf[e * W + col] = buf[r * W + col];
        buf[r * W + col] = t;
      }
    }
    __syncthreads();
    fft_smem(buf, n, logn, W, tw, true);
  }
  for (int q = threadIdx.x; q < n * W; q += blockDim.x) {
    int e = q / W, col = q % W;
    if (kz0 + col < hn) spec[base + e * es + kz0 + col] = buf[e * W + col];
  }
}

template <class R>
int cols_per_block(int n) {
  int w = kSmemBytes / (n * (int)sizeof(cplx<R>));
  if (w > 64) w = 64;
  if (w < 1) w = 1;
  return w;
}

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <class R>
void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_fft_z_r2c<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  cudaFuncSetAttribute(k_fft_z_c2r<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  cudaFuncSetAttribute(k_fft_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  done = true;
}

}  // namespace

// forward 3D r2c of an n^3 real array
template <class R>
void fft_r2c_3d(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw) {
  set_smem_attrs<R>();
  int logn = ilog2(n), W = cols_per_block<R>(n);
  int64_t npairs = (int64_t)n * n / 2;
  size_t sm = (size_t)n * W * sizeof(cplx<R>);
  k_fft_z_r2c<R><<<(unsigned)((npairs + W - 1) / W), kFftThreads, sm, c->stream>>>(in, out, n, logn, W, npairs, tw);
  int ncb = (n / 2 + 1 + W - 1) / W;
  k_fft_cols<R><<<n * ncb, kFftThreads, sm, c->stream>>>(out, n, logn, W, 1, 0, tw, nullptr, (R)0);
  k_fft_cols<R><<<n * ncb, kFftThreads, sm, c->stream>>>(out, n, logn, W, 0, 0, tw, nullptr, (R)0);
}

// inverse 3D c2r; when green != nullptr the X pass first runs forward and
// multiplies by the Green function (the spectrum then holds the Y/Z-forward
// data of the density and the X forward is fused here)
template <class R>
void fft_c2r_3d(dzs_ctx* c, cplx<R>* in, R* out, int n, const cplx<R>* tw, const R* green, R gfac) {
  set_smem_attrs<R>();
  int logn = ilog2(n), W = cols_per_block<R>(n);
  int64_t npairs = (int64_t)n * n / 2;
  size_t sm = (size_t)n * W * sizeof(cplx<R>);
  int ncb = (n / 2 + 1 + W - 1) / W;
  k_fft_cols<R><<<n * ncb, kFftThreads, sm, c->stream>>>(in, n, logn, W, 0, green ? 2 : 1, tw, green, gfac);
  k_fft_cols<R><<<n * ncb, kFftThreads, sm, c->stream>>>(in, n, logn, W, 1, 1, tw, nullptr, (R)0);
  k_fft_z_c2r<R><<<(unsigned)((npairs + W - 1) / W), kFftThreads, sm, c->stream>>>(in, out, n, logn, W, npairs, tw);
}

// forward Z and Y passes only (the X forward is fused with the Green multiply)
template <class R>
void fft_r2c_zy(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw) {
  set_smem_attrs<R>();
  int logn = ilog2(n), W = cols_per_block<R>(n);
  int64_t npairs = (int64_t)n * n / 2;
  size_t sm = (size_t)n * W * sizeof(cplx<R>);
  k_fft_z_r2c<R><<<(unsigned)((npairs + W - 1) / W), kFftThreads, sm, c->stream>>>(in, out, n, logn, W, npairs, tw);
  int ncb = (n / 2 + 1 + W - 1) / W;
  k_fft_cols<R><<<n * ncb, kFftThreads, sm, c->stream>>>(out, n, logn, W, 1, 0, tw, nullptr, (R)0);
}

template void fft_r2c_3d<float>(dzs_ctx*, const float*, cplx<float>*, int, const cplx<float>*);
template void fft_r2c_3d<double>(dzs_ctx*, const double*, cplx<double>*, int, const cplx<double>*);
template void fft_c2r_3d<float>(dzs_ctx*, cplx<float>*, float*, int, const cplx<float>*, const float*, float);
template void fft_c2r_3d<double>(dzs_ctx*, cplx<double>*, double*, int, const cplx<double>*, const double*, double);
template void fft_r2c_zy<float>(dzs_ctx*, const float*, cplx<float>*, int, const cplx<float>*);
template void fft_r2c_zy<double>(dzs_ctx*, const double*, cplx<double>*, int, const cplx<double>*);

// host twiddle table exp(-2 pi i t / n), t < n/2, in precision R
template <class R>
std::vector<cplx<R>> twiddles(int n) {
  std::vector<cplx<R>> t(n / 2 > 0 ? n / 2 : 1);
  for (int i = 0; i < n / 2; ++i) {
    double ang = -2.0 * M_PI * (double)i / (double)n;
    t[i] = {(R)std::cos(ang), (R)std::sin(ang)};
  }
  return t;
}
template std::vector<cplx<float>> twiddles<float>(int);
template std::vector<cplx<double>> twiddles<double>(int);

}  // namespace dzs
