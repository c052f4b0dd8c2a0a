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
// Each length-n transform is a four-step FFT, n = N1 N2 (n = 2^a, or 3 2^a
// with the factor 3 in N1; N2 a power of two): N2 register FFTs of length N1
// (input stride N2; a length 3 M register FFT is three length-M FFTs and
// radix-3 butterflies), twiddle W_n^(j2 k1),
// one exchange through shared memory, N1 register FFTs of length N2.  A thread
// owns one length-N1 and one length-N2 sub-transform of one column, so a
// column costs two register FFTs and one shared-memory round trip instead of
// log2(n) barrier-separated radix-2 stages.  Twiddles come from FP64 host
// tables (W_32 table in constant memory, W_n in global memory).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dzs {
namespace {

__constant__ cplx<float> kTw32f[32];   // exp(-2 pi i t / 32)
__constant__ cplx<double> kTw32d[32];
__constant__ cplx<float> kTw48f[48];   // exp(-2 pi i t / 48) (register FFTs of length 3 2^a <= 48)
__constant__ cplx<double> kTw48d[48];

__device__ __forceinline__ cplx<float> tw32(int t, float) { return kTw32f[t]; }
__device__ __forceinline__ cplx<double> tw32(int t, double) { return kTw32d[t]; }
__device__ __forceinline__ cplx<float> tw48(int t, float) { return kTw48f[t]; }
__device__ __forceinline__ cplx<double> tw48(int t, double) { return kTw48d[t]; }

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
constexpr int brevc(int v, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
  return r;
}

template <class R, int K>
__device__ __forceinline__ void reg_fft(cplx<R> (&a)[K], bool inv);

// length K = 3 M: three length-M FFTs of the residues mod 3, twiddles W_K^(r k),
// then for each k the radix-3 butterfly with w = exp(-+2 pi i / 3) = c + i s:
// X[k] = x0 + x1 + x2, X[k + M] = x0 + c (x1 + x2) + i s (x1 - x2),
// X[k + 2M] = x0 + c (x1 + x2) - i s (x1 - x2)
template <class R, int K>
__device__ __forceinline__ void reg_fft3(cplx<R> (&a)[K], bool inv) {
  constexpr int M = K / 3;
  cplx<R> s0[M], s1[M], s2[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    s0[j] = a[3 * j];
    s1[j] = a[3 * j + 1];
    s2[j] = a[3 * j + 2];
  }
  if (M > 1) {
    reg_fft<R, M>(s0, inv);
    reg_fft<R, M>(s1, inv);
    reg_fft<R, M>(s2, inv);
  }
  const R c = (R)-0.5;
  const R sn = inv ? (R)0.8660254037844386 : (R)-0.8660254037844386;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    cplx<R> w1 = tw48(k * (48 / K), R(0)), w2 = tw48((2 * k * (48 / K)) % 48, R(0));
    if (inv) {
      w1.y = -w1.y;
      w2.y = -w2.y;
    }
    const cplx<R> x0 = s0[k], x1 = cmul(s1[k], w1), x2 = cmul(s2[k], w2);
    const cplx<R> t1 = {x1.x + x2.x, x1.y + x2.y}, t2 = {x1.x - x2.x, x1.y - x2.y};
    const cplx<R> m = {x0.x + c * t1.x, x0.y + c * t1.y};
    a[k] = {x0.x + t1.x, x0.y + t1.y};
    a[k + M] = {m.x - sn * t2.y, m.y + sn * t2.x};
    a[k + 2 * M] = {m.x + sn * t2.y, m.y - sn * t2.x};
  }
}

// in-register FFT of length K (natural order in and out): radix-2 DIT for a
// power of two, reg_fft3 for 3 2^a; inv selects the conjugate twiddles
template <class R, int K>
__device__ __forceinline__ void reg_fft(cplx<R> (&a)[K], bool inv) {
  if constexpr (K % 3 == 0) {
    reg_fft3<R, K>(a, inv);
    return;
  }
  constexpr int L = ilog2c(K);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int j = brevc(i, L);
    if (j > i) {
      cplx<R> t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
#pragma unroll
  for (int s = 0; s < L; ++s) {
    const int half = 1 << s;
#pragma unroll
    for (int b = 0; b < K / 2; ++b) {
      const int j = b & (half - 1);
      const int i0 = ((b >> s) << (s + 1)) + j, i1 = i0 + half;
      cplx<R> w = tw32(j * (32 / (2 * half)), R(0));
      if (inv) w.y = -w.y;
      cplx<R> x = a[i0], y = cmul(a[i1], w);
      a[i0] = {x.x + y.x, x.y + y.y};
      a[i1] = {x.x - y.x, x.y - y.y};
    }
  }
}

// W_n^t from the half table tw[t] = exp(-2 pi i t / n), t < n / 2
template <class R>
__device__ __forceinline__ cplx<R> twn(const cplx<R>* __restrict__ tw, int t, int n, bool inv) {
  t %= n;  // n is a compile-time constant at every call (a mask for powers of two)
  cplx<R> w = t < n / 2 ? tw[t] : cplx<R>{-tw[t - n / 2].x, -tw[t - n / 2].y};
  if (inv) w.y = -w.y;
  return w;
}

template <int N>
struct Split {
  // powers of two: N1 = 2^ceil(a/2); N = 3 2^a: N2 = 2^floor(a/2), N1 = N / N2
  static constexpr int N2 = (N % 3 == 0) ? (1 << (ilog2c(N / 3) / 2)) : N / (1 << ((ilog2c(N) + 1) / 2));
  static constexpr int N1 = N / N2;
};

// shared-memory slot of element row `row` of column `col` in a block of W
// columns: for W a power of two the column index is XOR-swizzled with the row
// (the transposing loads of the Z passes, consecutive rows of one column, then
// fall on distinct banks; consecutive columns of one row stay a permutation of
// one row), otherwise rows are padded to W + 1
__device__ __forceinline__ int sidx(int row, int col, int W) {
  return (W & (W - 1)) == 0 ? row * W + (col ^ (row & (W - 1))) : row * (W + 1) + col;
}

__host__ __device__ constexpr int srows(int W) { return (W & (W - 1)) == 0 ? W : W + 1; }

// ---- generic four-step pieces on one column held in shared memory
// step A: thread (col, j2) transforms x[j1 N2 + j2] over j1, twiddles, and
// writes Y[k1 N2 + j2] back into the same column
template <class R, int N>
__device__ __forceinline__ void stepA_smem(cplx<R>* buf, int W, int col, int j2, const cplx<R>* __restrict__ tw,
                                           bool inv) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  cplx<R> a[N1];
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) a[j1] = buf[sidx((j1 * N2 + j2), col, W)];
  reg_fft<R, N1>(a, inv);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) a[k1] = cmul(a[k1], twn(tw, j2 * k1, N, inv));
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) buf[sidx((k1 * N2 + j2), col, W)] = a[k1];
}

// step B: thread (col, k1) transforms Y[k1 N2 + j2] over j2; result element
// k1 + N1 k2 is b[k2]
template <class R, int N>
__device__ __forceinline__ void stepB_smem(const cplx<R>* buf, int W, int col, int k1, cplx<R> (&b)[Split<N>::N2],
                                           bool inv) {
  constexpr int N2 = Split<N>::N2;
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) b[j2] = buf[sidx((k1 * N2 + j2), col, W)];
  reg_fft<R, N2>(b, inv);
}

// ---- Z pass, real -> half spectrum.  Block: W row pairs, W * N1 threads.
template <class R, int N>
__global__ void k_fft_z_r2c(const R* __restrict__ in, cplx<R>* __restrict__ out, int W, int64_t npairs,
                            const cplx<R>* __restrict__ tw) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, HN = N / 2 + 1;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw);
  const int64_t p0 = (int64_t)blockIdx.x * W;
  // coalesced load: element e of pair col at buf[sidx(e, col, W)]
  for (int q = threadIdx.x; q < N * W; q += blockDim.x) {
    int col = q / N, e = q % N;
    int64_t pr = p0 + col;
    cplx<R> v = {0, 0};
    if (pr < npairs) v = {in[(2 * pr) * N + e], in[(2 * pr + 1) * N + e]};
    buf[sidx(e, col, W)] = v;
  }
  __syncthreads();
  const int col = threadIdx.x % W, r = threadIdx.x / W;
  if (r < N2) stepA_smem<R, N>(buf, W, col, r, tw, false);
  __syncthreads();
  cplx<R> b[N2];
  if (r < N1) stepB_smem<R, N>(buf, W, col, r, b, false);
  __syncthreads();
  if (r < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) buf[sidx((r + N1 * k2), col, W)] = b[k2];
  }
  __syncthreads();
  // unpack: X_a = (Z_k + conj Z_-k) / 2,  X_b = (Z_k - conj Z_-k) / (2 i)
  for (int q = threadIdx.x; q < HN * W; q += blockDim.x) {
    int c = q / HN, k = q % HN;
    int64_t pr = p0 + c;
    if (pr >= npairs) continue;
    cplx<R> z = buf[sidx((k % N), c, W)], zc = buf[sidx(((N - k) % N), c, W)];
    out[(2 * pr) * HN + k] = {(R)0.5 * (z.x + zc.x), (R)0.5 * (z.y - zc.y)};
    out[(2 * pr + 1) * HN + k] = {(R)0.5 * (z.y + zc.y), (R)-0.5 * (z.x - zc.x)};
  }
}

// ---- Z pass inverse, half spectrum -> real (unnormalised).
template <class R, int N>
__global__ void k_fft_z_c2r(const cplx<R>* __restrict__ in, R* __restrict__ out, int W, int64_t npairs,
                            const cplx<R>* __restrict__ tw) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, HN = N / 2 + 1;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw);
  const int64_t p0 = (int64_t)blockIdx.x * W;
  for (int q = threadIdx.x; q < N * W; q += blockDim.x) {
    int col = q / N, k = q % N;
    int64_t pr = p0 + col;
    cplx<R> z = {0, 0};
    if (pr < npairs) {
      cplx<R> a, b;
      if (k < HN) {
        a = in[(2 * pr) * HN + k];
        b = in[(2 * pr + 1) * HN + k];
      } else {
        a = in[(2 * pr) * HN + (N - k)];
        b = in[(2 * pr + 1) * HN + (N - k)];
        a.y = -a.y;
        b.y = -b.y;
      }
      z = {a.x - b.y, a.y + b.x};  // a + i b
    }
    buf[sidx(k, col, W)] = z;
  }
  __syncthreads();
  const int col = threadIdx.x % W, r = threadIdx.x / W;
  if (r < N2) stepA_smem<R, N>(buf, W, col, r, tw, true);
  __syncthreads();
  cplx<R> b[N2];
  if (r < N1) stepB_smem<R, N>(buf, W, col, r, b, true);
  __syncthreads();
  if (r < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) buf[sidx((r + N1 * k2), col, W)] = b[k2];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < N * W; q += blockDim.x) {
    int c = q / N, e = q % N;
    int64_t pr = p0 + c;
    if (pr >= npairs) continue;
    cplx<R> z = buf[sidx(e, c, W)];
    out[(2 * pr) * N + e] = z.x;
    out[(2 * pr + 1) * N + e] = z.y;
  }
}

// ---- column pass along Y (axis 1) or X (axis 0) of the half spectrum.
// mode 0 forward, 1 inverse, 2 forward + Green multiply + inverse (X only).
// Block: one line (ix for Y, iy for X) and W consecutive kz columns.
template <class R, int N>
__global__ void k_fft_cols(cplx<R>* __restrict__ spec, int W, int axis, int mode, const cplx<R>* __restrict__ tw,
                           const R* __restrict__ gtab, R gfac) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, HN = N / 2 + 1;
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* buf = reinterpret_cast<cplx<R>*>(smem_raw);
  const int ncb = (HN + W - 1) / W;
  const int line = blockIdx.x / ncb;
  const int kz0 = (blockIdx.x % ncb) * W;
  const int64_t es = axis == 1 ? (int64_t)HN : (int64_t)N * HN;
  const int64_t base = axis == 1 ? (int64_t)line * N * HN : (int64_t)line * HN;
  const int col = threadIdx.x % W, r = threadIdx.x / W;
  const bool valid = kz0 + col < HN;
  const bool inv = mode == 1;
  // step A straight from global memory (coalesced across columns)
  if (r < N2) {
    cplx<R> a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) a[j1] = valid ? spec[base + (j1 * N2 + r) * es + kz0 + col] : cplx<R>{0, 0};
    reg_fft<R, N1>(a, inv);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[sidx((k1 * N2 + r), col, W)] = cmul(a[k1], twn(tw, r * k1, N, inv));
  }
  __syncthreads();
  cplx<R> b[N2];
  if (r < N1) stepB_smem<R, N>(buf, W, col, r, b, inv);
  if (mode != 2) {
    if (r < N1 && valid) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) spec[base + (r + N1 * k2) * es + kz0 + col] = b[k2];
    }
    return;
  }
  // Green multiply on element kx = r + N1 k2 (gtab: per-axis k^2, W_CIC, r_s^2)
  const R* k2t = gtab;
  const R* wt = gtab + N;
  const int kz = kz0 + col;
  if (r < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int kx = r + N1 * k2;
      R gv = 0;
      if (valid) {
        R kk = k2t[kx] + k2t[line] + k2t[kz];
        if (kk > (R)0) {
          R wv = wt[kx] * wt[line] * wt[kz];
          gv = gfac * exp(-kk * gtab[2 * N]) / (kk * wv * wv);
        }
      }
      b[k2] = {b[k2].x * gv, b[k2].y * gv};
    }
  }
  // inverse with the roles of N1 and N2 swapped: this thread holds the
  // elements r + N1 k2, i.e. one length-N2 sub-sequence of stride N1
  __syncthreads();
  if (r < N1) {
    reg_fft<R, N2>(b, true);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) buf[sidx((k2 * N1 + r), col, W)] = cmul(b[k2], twn(tw, r * k2, N, true));
  }
  __syncthreads();
  if (r < N2) {
    cplx<R> a[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) a[j] = buf[sidx((r * N1 + j), col, W)];
    reg_fft<R, N1>(a, true);
    if (valid) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) spec[base + (r + N2 * k1) * es + kz0 + col] = a[k1];
    }
  }
}

template <class R, int N>
int cols_per_block() {
  // W * N1 threads per block, at most 256; shared memory srows(W) * N * sizeof(cplx)
  int w = 256 / Split<N>::N1;
  while (w > 1 && (size_t)srows(w) * N * sizeof(cplx<R>) > 48 * 1024) w >>= 1;
  return w;
}

template <class R, int N>
void launch_r2c_zy(dzs_ctx* c, const R* in, cplx<R>* out, const cplx<R>* tw, bool do_x) {
  const int W = cols_per_block<R, N>();
  const int threads = W * Split<N>::N1;
  const size_t sm = (size_t)N * srows(W) * sizeof(cplx<R>);
  const int64_t npairs = (int64_t)N * N / 2;
  k_fft_z_r2c<R, N><<<(unsigned)((npairs + W - 1) / W), threads, sm, c->stream>>>(in, out, W, npairs, tw);
  const int ncb = (N / 2 + 1 + W - 1) / W;
  k_fft_cols<R, N><<<N * ncb, threads, sm, c->stream>>>(out, W, 1, 0, tw, nullptr, (R)0);
  if (do_x) k_fft_cols<R, N><<<N * ncb, threads, sm, c->stream>>>(out, W, 0, 0, tw, nullptr, (R)0);
}

template <class R, int N>
void launch_c2r(dzs_ctx* c, cplx<R>* in, R* out, const cplx<R>* tw, const R* green, R gfac) {
  const int W = cols_per_block<R, N>();
  const int threads = W * Split<N>::N1;
  const size_t sm = (size_t)N * srows(W) * sizeof(cplx<R>);
  const int64_t npairs = (int64_t)N * N / 2;
  const int ncb = (N / 2 + 1 + W - 1) / W;
  k_fft_cols<R, N><<<N * ncb, threads, sm, c->stream>>>(in, W, 0, green ? 2 : 1, tw, green, gfac);
  k_fft_cols<R, N><<<N * ncb, threads, sm, c->stream>>>(in, W, 1, 1, tw, nullptr, (R)0);
  k_fft_z_c2r<R, N><<<(unsigned)((npairs + W - 1) / W), threads, sm, c->stream>>>(in, out, W, npairs, tw);
}

template <class R>
void dispatch_r2c(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw, bool do_x) {
  switch (n) {
    case 8: launch_r2c_zy<R, 8>(c, in, out, tw, do_x); break;
    case 16: launch_r2c_zy<R, 16>(c, in, out, tw, do_x); break;
    case 32: launch_r2c_zy<R, 32>(c, in, out, tw, do_x); break;
    case 64: launch_r2c_zy<R, 64>(c, in, out, tw, do_x); break;
    case 128: launch_r2c_zy<R, 128>(c, in, out, tw, do_x); break;
    case 256: launch_r2c_zy<R, 256>(c, in, out, tw, do_x); break;
    case 512: launch_r2c_zy<R, 512>(c, in, out, tw, do_x); break;
    case 12: launch_r2c_zy<R, 12>(c, in, out, tw, do_x); break;
    case 24: launch_r2c_zy<R, 24>(c, in, out, tw, do_x); break;
    case 48: launch_r2c_zy<R, 48>(c, in, out, tw, do_x); break;
    case 96: launch_r2c_zy<R, 96>(c, in, out, tw, do_x); break;
    case 192: launch_r2c_zy<R, 192>(c, in, out, tw, do_x); break;
    case 384: launch_r2c_zy<R, 384>(c, in, out, tw, do_x); break;
    default: break;  // sizes are validated at context creation
  }
}

template <class R>
void dispatch_c2r(dzs_ctx* c, cplx<R>* in, R* out, int n, const cplx<R>* tw, const R* green, R gfac) {
  switch (n) {
    case 8: launch_c2r<R, 8>(c, in, out, tw, green, gfac); break;
    case 16: launch_c2r<R, 16>(c, in, out, tw, green, gfac); break;
    case 32: launch_c2r<R, 32>(c, in, out, tw, green, gfac); break;
    case 64: launch_c2r<R, 64>(c, in, out, tw, green, gfac); break;
    case 128: launch_c2r<R, 128>(c, in, out, tw, green, gfac); break;
    case 256: launch_c2r<R, 256>(c, in, out, tw, green, gfac); break;
    case 512: launch_c2r<R, 512>(c, in, out, tw, green, gfac); break;
    case 12: launch_c2r<R, 12>(c, in, out, tw, green, gfac); break;
    case 24: launch_c2r<R, 24>(c, in, out, tw, green, gfac); break;
    case 48: launch_c2r<R, 48>(c, in, out, tw, green, gfac); break;
    case 96: launch_c2r<R, 96>(c, in, out, tw, green, gfac); break;
    case 192: launch_c2r<R, 192>(c, in, out, tw, green, gfac); break;
    case 384: launch_c2r<R, 384>(c, in, out, tw, green, gfac); break;
    default: break;
  }
}

}  // namespace

// forward 3D r2c of an n^3 real array
template <class R>
void fft_r2c_3d(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw) {
  dispatch_r2c<R>(c, in, out, n, tw, true);
}

// inverse 3D c2r; when green != nullptr the X pass runs forward, multiplies by
// the Green function and runs inverse (the spectrum then holds the Z/Y-forward
// data of the density)
template <class R>
void fft_c2r_3d(dzs_ctx* c, cplx<R>* in, R* out, int n, const cplx<R>* tw, const R* green, R gfac) {
  dispatch_c2r<R>(c, in, out, n, tw, green, gfac);
}

// forward Z and Y passes only (the X forward is fused with the Green multiply)
template <class R>
void fft_r2c_zy(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw) {
  dispatch_r2c<R>(c, in, out, n, tw, false);
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

// the length-32 and length-48 register-FFT tables in constant memory (both precisions)
void upload_fft_constants(int dev) {
  static bool done[256] = {false};
  if (dev < 0 || dev >= 256 || done[dev]) return;
  cplx<float> tf[32];
  cplx<double> td[32];
  for (int t = 0; t < 32; ++t) {
    double ang = -2.0 * M_PI * (double)t / 32.0;
    td[t] = {std::cos(ang), std::sin(ang)};
    tf[t] = {(float)td[t].x, (float)td[t].y};
  }
  cudaMemcpyToSymbol(kTw32f, tf, sizeof tf);
  cudaMemcpyToSymbol(kTw32d, td, sizeof td);
  cplx<float> tf48[48];
  cplx<double> td48[48];
  for (int t = 0; t < 48; ++t) {
    double ang = -2.0 * M_PI * (double)t / 48.0;
    td48[t] = {std::cos(ang), std::sin(ang)};
    tf48[t] = {(float)td48[t].x, (float)td48[t].y};
  }
  cudaMemcpyToSymbol(kTw48f, tf48, sizeof tf48);
  cudaMemcpyToSymbol(kTw48d, td48, sizeof td48);
  done[dev] = true;
}

}  // namespace dzs
