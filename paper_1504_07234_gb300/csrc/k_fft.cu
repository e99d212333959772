// k_fft.cu — the regularising preconditioners of Sections 4 and 5 applied
// through batched two-pass 2-D transforms.
//
//   t = T^{-1} [ w(k) * T r ]      (T = 2-D DFT or 2-D DCT-II)
//   w = 1/(sigma + alpha)          (Eq. Alg1, Alg3; M in Algorithm 2)
//   w = conj(lambda)/(sigma+alpha) (Eq. Alg4, Algorithm 4-NS)
//
// Pass 1 (rows): two real rows are packed into one complex FFT; DFT keeps the
// half spectrum, DCT-II uses the even/odd reordering of the input so that
// X[k] = Re(exp(-i pi k / 2n) V[k]) with V the DFT of the reordered row.
// Pass 2 (columns): forward, weight, inverse on columns held in shared memory
// (for 4-NS the forward spectrum is kept for the alpha_n solve and the weight
// and inverse run after it).  Pass 3 (rows): inverse.  The unnormalised
// forward / inverse pair gives n^2 times the result; 1/n^2 is folded into the
// weight.  Weights are formed in T from |lambda|^2 rounded once to T.
//
// The spectrum (S, lambda, |lambda|^2) is stored column-blocked: columns are
// grouped in blocks of cb, each block n rows x cb contiguous elements, so a
// column-pass CTA reads and writes one contiguous block and the row passes
// write / read contiguous runs of cb.
//
// The 1-D FFT is a Stockham autosort FFT in shared memory with radix 16, 8,
// 4, 2, 3 and 5 passes (16 and 8 as 4 x 4 and 4 x 2 register butterflies with
// constant inner twiddles); each pass loads all butterfly inputs of a thread
// into registers, synchronises, and stores in place.  Shared memory holds
// element i of a transform at i + i/16 so that radix-R strides do not hit the
// same bank.
#include "mlba_internal.cuh"
#include "mlba_launch.h"

namespace mlba {

// ---------------------------------------------------------------------------
// small DFTs (forward: exp(-2 pi i jk/R); INV: conjugate)
template <typename T2, bool INV>
__device__ __forceinline__ void dft2(T2* v) {
  T2 a = v[0], b = v[1];
  v[0] = cadd(a, b); v[1] = csub(a, b);
}
template <typename T2, bool INV>
__device__ __forceinline__ void dft4(T2* v) {
  T2 a = v[0], b = v[1], c = v[2], d = v[3];
  T2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
  // -i * s3 (forward) or +i * s3 (inverse)
  T2 js3;
  if (INV) { js3.x = -s3.y; js3.y = s3.x; } else { js3.x = s3.y; js3.y = -s3.x; }
  v[0] = cadd(s0, s2); v[2] = csub(s0, s2);
  v[1] = cadd(s1, js3); v[3] = csub(s1, js3);
}
template <typename T2, bool INV>
__device__ __forceinline__ void dft3(T2* v) {
  using T = decltype(v[0].x);
  const T h = T(0.86602540378443864676);   // sin(2 pi / 3)
  T2 a = v[0], b = v[1], c = v[2];
  T2 t1 = cadd(b, c), t2 = csub(b, c);
  T2 m; m.x = a.x - T(0.5) * t1.x; m.y = a.y - T(0.5) * t1.y;
  // forward: X1 = m - i h t2, X2 = m + i h t2
  T2 ih; ih.x = -h * t2.y; ih.y = h * t2.x;   // i h t2
  v[0] = cadd(a, t1);
  if (INV) { v[1] = cadd(m, ih); v[2] = csub(m, ih); }
  else { v[1] = csub(m, ih); v[2] = cadd(m, ih); }
}
template <typename T2, bool INV>
__device__ __forceinline__ void dft5(T2* v) {
  using T = decltype(v[0].x);
  const T c1 = T(0.30901699437494742410);   // cos(2 pi/5)
  const T c2 = T(-0.80901699437494742410);  // cos(4 pi/5)
  const T s1 = T(0.95105651629515357212);   // sin(2 pi/5)
  const T s2 = T(0.58778525229247312917);   // sin(4 pi/5)
  T2 a = v[0];
  T2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  T2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  T2 m1, m2, n1, n2;
  m1.x = a.x + c1 * t1.x + c2 * t2.x; m1.y = a.y + c1 * t1.y + c2 * t2.y;
  m2.x = a.x + c2 * t1.x + c1 * t2.x; m2.y = a.y + c2 * t1.y + c1 * t2.y;
  // n1 = s1 t3 + s2 t4 ; n2 = s2 t3 - s1 t4
  n1.x = s1 * t3.x + s2 * t4.x; n1.y = s1 * t3.y + s2 * t4.y;
  n2.x = s2 * t3.x - s1 * t4.x; n2.y = s2 * t3.y - s1 * t4.y;
  // i * n
  T2 in1, in2; in1.x = -n1.y; in1.y = n1.x; in2.x = -n2.y; in2.y = n2.x;
  v[0] = cadd(a, cadd(t1, t2));
  if (INV) {
    v[1] = cadd(m1, in1); v[4] = csub(m1, in1);
    v[2] = cadd(m2, in2); v[3] = csub(m2, in2);
  } else {
    v[1] = csub(m1, in1); v[4] = cadd(m1, in1);
    v[2] = csub(m2, in2); v[3] = cadd(m2, in2);
  }
}
// cos and sin of 2 pi m / 16 for the inner twiddles of the radix-16 and
// radix-8 butterflies (m < 16)
__host__ __device__ constexpr double cos16(int m) {
  return m == 0 ? 1.0 : m == 1 ? 0.92387953251128675613 : m == 2 ? 0.70710678118654752440
       : m == 3 ? 0.38268343236508977173 : m == 4 ? 0.0 : m == 5 ? -0.38268343236508977173
       : m == 6 ? -0.70710678118654752440 : m == 7 ? -0.92387953251128675613 : m == 8 ? -1.0
       : -cos16(m - 8);
}
__host__ __device__ constexpr double sin16(int m) { return cos16((m + 12) % 16); }
// multiply by exp(-/+ 2 pi i m / 16) for a compile-time m
template <typename T2, int M, bool INV>
__device__ __forceinline__ T2 tw16(T2 a) {
  using T = decltype(a.x);
  if (M % 16 == 0) return a;
  const T cr = T(cos16(M % 16)), si = INV ? T(sin16(M % 16)) : T(-sin16(M % 16));
  T2 r; r.x = a.x * cr - a.y * si; r.y = a.x * si + a.y * cr;
  return r;
}
// 16-point DFT as 4 x 4: X[k1 + 4 k2] = sum_r1 w4^(r1 k2) [w16^(r1 k1) DFT4_r2(v[r1 + 4 r2])](k1)
template <typename T2, bool INV>
__device__ __forceinline__ void dft16(T2* v) {
  T2 y[4][4];
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) {
    T2 a[4] = {v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]};
    dft4<T2, INV>(a);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[r1][k1] = a[k1];
  }
  y[1][1] = tw16<T2, 1, INV>(y[1][1]); y[1][2] = tw16<T2, 2, INV>(y[1][2]); y[1][3] = tw16<T2, 3, INV>(y[1][3]);
  y[2][1] = tw16<T2, 2, INV>(y[2][1]); y[2][2] = tw16<T2, 4, INV>(y[2][2]); y[2][3] = tw16<T2, 6, INV>(y[2][3]);
  y[3][1] = tw16<T2, 3, INV>(y[3][1]); y[3][2] = tw16<T2, 6, INV>(y[3][2]); y[3][3] = tw16<T2, 9, INV>(y[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    T2 b[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
    dft4<T2, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}
// 8-point DFT as 4 x 2: X[k1 + 4 k2] = sum_r1 w2^(r1 k2) [w8^(r1 k1) DFT4_r2(v[r1 + 2 r2])](k1)
template <typename T2, bool INV>
__device__ __forceinline__ void dft8(T2* v) {
  T2 y[2][4];
#pragma unroll
  for (int r1 = 0; r1 < 2; ++r1) {
    T2 a[4] = {v[r1], v[r1 + 2], v[r1 + 4], v[r1 + 6]};
    dft4<T2, INV>(a);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[r1][k1] = a[k1];
  }
  y[1][1] = tw16<T2, 2, INV>(y[1][1]); y[1][2] = tw16<T2, 4, INV>(y[1][2]); y[1][3] = tw16<T2, 6, INV>(y[1][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    T2 b[2] = {y[0][k1], y[1][k1]};
    dft2<T2, INV>(b);
    v[k1] = b[0];
    v[k1 + 4] = b[1];
  }
}

template <typename T2, int R, bool INV>
__device__ __forceinline__ void dft_small(T2* v) {
  if (R == 2) dft2<T2, INV>(v);
  else if (R == 3) dft3<T2, INV>(v);
  else if (R == 4) dft4<T2, INV>(v);
  else if (R == 5) dft5<T2, INV>(v);
  else if (R == 8) dft8<T2, INV>(v);
  else dft16<T2, INV>(v);
}

// threads of a transform CTA and the minimum CTAs per SM (register budget):
// FP32 256 threads, at least 4 CTAs (64 registers: a few spilled values cost
// less than the lost overlap of the barrier-separated phases at 3 CTAs per
// SM); FP64 512 threads, so that each thread holds half as many values
__host__ __device__ constexpr int tr_nt(int elem_bytes) { return elem_bytes == 8 ? 512 : 256; }
__host__ __device__ constexpr int tr_minb(int elem_bytes) { return elem_bytes == 8 ? 1 : 4; }

// shared-memory layout of a transform: element i at fpad(i) (one spare slot
// every 16 breaks power-of-two strides), transforms TSg = fpad(N) + 1 apart
__host__ __device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

// One Stockham pass of radix R over G transforms of length N.  Each thread
// loads all inputs of its butterflies, the block synchronises, then stores:
// the pass runs in place.
template <typename T2, int R, bool INV>
__device__ __forceinline__ void fft_pass(int G, int N, int TSg, int Ns, const T2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  constexpr int NT = tr_nt(sizeof(T2) / 2);
  constexpr int MAXB = (TR_CAP + R * NT - 1) / (R * NT);
  const int per = N / R;
  const int nbf = G * per;
  const int step = N / (Ns * R);
  const FastDiv fper(per), fns(Ns);
  T2 v[MAXB][R];
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * NT;
    if (b < nbf) {
      const int g = fper.div(b), j = b - g * per;
      const int k = j - fns.div(j) * Ns;
      const T2* base = sm + g * TSg;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = base[fpad(j + r * per)];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          T2 w = __ldg(&tw[r * k * step]);
          if (INV) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft_small<T2, R, INV>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * NT;
    if (b < nbf) {
      const int g = fper.div(b), j = b - g * per;
      const int jd = fns.div(j);
      const int k = j - jd * Ns;
      T2* base = sm + g * TSg;
      const int o = jd * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) base[fpad(o + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// One Stockham pass of any radix R (the prime factors of n above 5) over G
// transforms of length N, as a direct sum: output s of butterfly j is
//   sum_r x[j + r N/R] exp(-/+ 2 pi i (r k step + ((r s) mod R) N/R) / N)
// with k = j mod Ns, step = N/(Ns R): the Stockham twiddle of input r and the
// R-point DFT kernel folded into one index of the length-N table.  Each
// thread computes whole outputs (R complex multiply-adds each, O(N R) per
// pass) and holds them in registers until the block has read its inputs.
template <typename T2, bool INV>
__device__ __noinline__ void fft_pass_any(int G, int N, int TSg, int Ns, int R,
                                          const T2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  constexpr int NT = tr_nt(sizeof(T2) / 2);
  constexpr int MAXO = TR_CAP / NT;
  const int per = N / R, step = N / (Ns * R);
  const FastDiv fN(N), fR(R), fns(Ns);
  T2 out[MAXO];
#pragma unroll
  for (int q = 0; q < MAXO; ++q) {
    const int e = threadIdx.x + q * NT;
    out[q].x = out[q].y = 0;
    if (e < G * N) {
      const int g = fN.div(e), rem = e - g * N;
      const int j = fR.div(rem), sidx = rem - j * R;
      const int k = j - fns.div(j) * Ns;
      const T2* base = sm + g * TSg;
      const int ks = k * step;
      int rs = 0;                     // (r s) mod R, advanced by s each term
      T2 acc = base[fpad(j)];         // r = 0: no twiddle
      for (int r = 1; r < R; ++r) {
        rs += sidx; if (rs >= R) rs -= R;
        int ti = r * ks + rs * per;   // < 2N
        if (ti >= N) ti -= N;
        T2 w = __ldg(&tw[ti]);
        if (INV) w.y = -w.y;
        const T2 v = base[fpad(j + r * per)];
        acc.x += v.x * w.x - v.y * w.y;
        acc.y += v.x * w.y + v.y * w.x;
      }
      out[q] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MAXO; ++q) {
    const int e = threadIdx.x + q * NT;
    if (e < G * N) {
      const int g = fN.div(e), rem = e - g * N;
      const int j = fR.div(rem), sidx = rem - j * R;
      const int jd = fns.div(j), k = j - jd * Ns;
      sm[g * TSg + fpad(jd * Ns * R + k + sidx * Ns)] = out[q];
    }
  }
  __syncthreads();
}

// G transforms of length n held in the dynamic shared memory of the block
// (transform g at g * (fpad(n) + 1)); all threads of the block call this
// The passes run grouped by radix (16s, one 8/4/2, 3s, 5s) in straight-line
// regions rather than as one loop over a radix switch: the compiler then
// keeps each region's butterflies in registers (the switch form spilled).
template <typename T2, bool INV>
__device__ __noinline__ void fft_smem(int G, const Prob& pd) {
  const int N = pd.nfft;
  const int TSg = fpad(N) + 1;
  const T2* tw = static_cast<const T2*>(pd.tw);
  const int n16 = pd.nr16, r2 = pd.r2, n3 = pd.nr3, n5 = pd.nr5;
  int Ns = 1;
  for (int s = 0; s < n16; ++s) { fft_pass<T2, 16, INV>(G, N, TSg, Ns, tw); Ns *= 16; }
  if (r2 == 8) { fft_pass<T2, 8, INV>(G, N, TSg, Ns, tw); Ns *= 8; }
  if (r2 == 4) { fft_pass<T2, 4, INV>(G, N, TSg, Ns, tw); Ns *= 4; }
  if (r2 == 2) { fft_pass<T2, 2, INV>(G, N, TSg, Ns, tw); Ns *= 2; }
  for (int s = 0; s < n3; ++s) { fft_pass<T2, 3, INV>(G, N, TSg, Ns, tw); Ns *= 3; }
  for (int s = 0; s < n5; ++s) { fft_pass<T2, 5, INV>(G, N, TSg, Ns, tw); Ns *= 5; }
  // prime factors above 5 (the plan lists them after the smooth passes)
  for (int s = pd.nstage - pd.nrany; s < pd.nstage; ++s) {
    const int R = pd.radix[s];
    fft_pass_any<T2, INV>(G, N, TSg, Ns, R, tw);
    Ns *= R;
  }
}

// position of input sample y in the DCT reordering v[j] = x[2j], v[N-1-j] = x[2j+1]
__device__ __forceinline__ int dct_pos(int y, int N) {
  return (y & 1) ? N - 1 - (y >> 1) : (y >> 1);
}
// inverse: sample stored at position j of v
__device__ __forceinline__ int dct_src(int j, int N) {
  return (j < (N + 1) / 2) ? 2 * j : 2 * (N - 1 - j) + 1;
}

// After a forward FFT of (a + i b) (two reordered real sequences): DCT-II of
// both, X[k] = Re(exp(-i pi k/2N) V[k]); results stored as (Xa, Xb) at k.
// Positions k and N-k depend only on each other, so one thread owns the pair
// and updates it in place.
template <typename T, typename T2>
__device__ __forceinline__ T2 split_one(T2 Z, T2 Zr, T2 d) {
  // Va = (Z + conj Zr)/2, Vb = (Z - conj Zr)/(2i), X = Re(d V)
  T2 va, vb, o;
  va.x = T(0.5) * (Z.x + Zr.x); va.y = T(0.5) * (Z.y - Zr.y);
  vb.x = T(0.5) * (Z.y + Zr.y); vb.y = T(-0.5) * (Z.x - Zr.x);
  o.x = d.x * va.x - d.y * va.y;
  o.y = d.x * vb.x - d.y * vb.y;
  return o;
}
template <typename T, typename T2>
__device__ __forceinline__ void dct_split(T2* sm, int G, int N, int TSg, const T2* __restrict__ dtw) {
  constexpr int NT = tr_nt(sizeof(T));
  const int np = N / 2 + 1;
  const FastDiv fnp(np);
  for (int e = threadIdx.x; e < G * np; e += NT) {
    const int g = fnp.div(e), k = e - g * np;
    const int kr = (k == 0) ? 0 : N - k;
    T2* b = sm + g * TSg;
    const T2 Z = b[fpad(k)], Zr = b[fpad(kr)];
    const T2 ok = split_one<T, T2>(Z, Zr, __ldg(&dtw[k]));
    if (kr != k) b[fpad(kr)] = split_one<T, T2>(Zr, Z, __ldg(&dtw[kr]));
    b[fpad(k)] = ok;
  }
  __syncthreads();
}

// Inverse of dct_split: from (Xa, Xb) at k build Z = Va + i Vb with
// V[k] = exp(+i pi k/2N) (X[k] - i X[N-k]), X[N] = 0, ready for an inverse FFT.
template <typename T, typename T2>
__device__ __forceinline__ T2 merge_one(T2 X, T2 Xr, T2 d) {
  d.y = -d.y;                               // exp(+i pi k/2N)
  T2 wa, wb;
  wa.x = X.x; wa.y = -Xr.x;
  wb.x = X.y; wb.y = -Xr.y;
  const T2 va = cmul(d, wa), vb = cmul(d, wb);
  T2 o; o.x = va.x - vb.y; o.y = va.y + vb.x;   // Va + i Vb
  return o;
}
template <typename T, typename T2>
__device__ __forceinline__ void dct_merge(T2* sm, int G, int N, int TSg, const T2* __restrict__ dtw) {
  constexpr int NT = tr_nt(sizeof(T));
  const int np = N / 2 + 1;
  const FastDiv fnp(np);
  for (int e = threadIdx.x; e < G * np; e += NT) {
    const int g = fnp.div(e), k = e - g * np;
    T2* b = sm + g * TSg;
    const T2 X = b[fpad(k)];
    T2 Xr;
    if (k == 0) { Xr.x = T(0); Xr.y = T(0); } else Xr = b[fpad(N - k)];
    const T2 ok = merge_one<T, T2>(X, Xr, __ldg(&dtw[k]));
    if (k != 0 && N - k != k) b[fpad(N - k)] = merge_one<T, T2>(Xr, X, __ldg(&dtw[N - k]));
    b[fpad(k)] = ok;
  }
  __syncthreads();
}

__device__ __forceinline__ bool tr_skip(const State& st, int pcg) {
  return st.stopped || (pcg && st.pdone);
}

// ---------------------------------------------------------------------------
// Algorithm 4-NS: alpha_n of Eq. Alg4_rev_7.  With a unitary transform the
// equation reads h(b) = F(a)/P - q_n^2 = 0, a = exp(b), P = sum |r^|^2,
// F(a) = sum |r^|^2 x^2, x = a/(s+a).  h increases with b (unique root);
// with dx/db = x(1-x) its derivatives are
//   h'  = 2 sum |r^|^2 x^2 (1-x) / P,
//   h'' = 2 sum |r^|^2 x^2 (1-x)(2-3x) / P.
// The spectrum in S is the unnormalised one; every coefficient carries its
// orthonormal weight, so the ratio is exact.  Pass 1 evaluates h and h' at
// NS_CAND points b_prev + (j - (NS_CAND - 1)/2) NS_CAND_STEP (a window of
// +-7 around the previous root), brackets the root and takes the root of the
// cubic Hermite interpolant on the bracket.  Later
// passes take safeguarded Halley steps inside the bracket; a step below
// tol, or below ns_tol3 (the next error is of the order of its cube), ends
// the solve.  Each block sums its share in T precision (FP64 across
// blocks); the last block updates the scalar state.
// 8 candidates 2 apart: the candidate sums are the bulk of the bracketing
// pass, and the wider Hermite bracket costs at most one more Halley pass
// (FP32: 2 of the 3 in the step, FP64: 3 of 5 on the workloads' spectra)
constexpr int NS_CAND = 8;
constexpr double NS_CAND_STEP = 2.0;
constexpr int NS_NT = SPEC_THREADS, NS_PT = SPEC_PER_THREAD;
constexpr int NS_B = 8;                    // elements per thread with loads in flight together
static_assert(NS_PT % NS_B == 0, "spectrum pass batches");
static_assert(SPEC_SUMS == 2 * NS_CAND + 1, "partial buffer sized for the bracketing pass");

__host__ __device__ constexpr double ns_tol(int elem_bytes) { return elem_bytes == 8 ? 1e-10 : 1e-5; }
// FP32: cbrt(tol) / 8, where the error after a Halley step (of the order of
// the step's cube) is far below tol; FP64 takes only steps below tol
__host__ __device__ constexpr double ns_tol3(int elem_bytes) { return elem_bytes == 8 ? 1e-10 : 2.7e-3; }

// element e (< NS_NT * NS_PT) of spectrum block `blk`, enumerated along the
// column-blocked layout (contiguous reads): weighted power and |lambda|^2 in
// T precision; false past the end or on padding
template <typename T>
__device__ __forceinline__ bool spec_elem(const Prob& pd, int blk, int e, T& pw, T& sg) {
  using T2 = typename Vec2<T>::type;
  const int N = pd.n, cb = pd.cb;
  const bool dct = (pd.transform == TR_DCT);
  const int W = dct ? N : pd.half;
  const int L = blk * (NS_NT * NS_PT) + e;      // < 2^31: one spectrum holds < 2^25 elements
  const int blksz = N * cb;
  const int b = L / blksz;
  const int rem = L - b * blksz;
  // rem < 2 TR_CAP and cb <= 2 TR_CAP: rem * cb < 2^32, the multiply-high
  // quotient is exact
  const int k1 = FastDiv(cb).div(rem), c = rem - k1 * cb;
  const int k2 = b * cb + c;
  if (k2 >= W) return false;
  if (dct) {
    // unnormalised DCT-II: |orthonormal coefficient|^2 = v^2 s_k1^2 s_k2^2
    // with s_0^2 = 1/N and s_k^2 = 2/N; the common 1/N^2 cancels
    const T v = static_cast<const T*>(pd.buf[SL_S])[L];
    pw = T((k1 == 0 ? 1 : 2) * (k2 == 0 ? 1 : 2)) * v * v;
  } else {
    const T2 v = static_cast<const T2*>(pd.buf[SL_S])[L];
    const T m = (k2 == 0 || ((N & 1) == 0 && k2 == N / 2)) ? T(1) : T(2);
    pw = m * (v.x * v.x + v.y * v.y);
  }
  sg = static_cast<const T*>(pd.w)[L];
  return true;
}

__device__ __forceinline__ void ns_set_alpha(const Prob& pd, State& st, double nb) {
  if (nb < -32.2) nb = -32.2;                          // alpha floor 1e-14
  st.nb = nb;
  double a = exp(nb);
  st.ea = a;
  if (pd.bc == BC_RECT && a < pd.alpha) a = pd.alpha;  // rectangular hybrid floor
  st.alpha_n = a;
  const int it = st.iter - 1;
  if (it >= 0 && it < pd.max_iter + 2) pd.hist_alpha[it] = a;
}

// Block totals of K values of type A (the warp sums stay in A: FP32 for the
// FP32 path, where FP64 arithmetic is scarce), then the cross-warp and
// cross-block totals in FP64 in the block that arrives last (true there;
// tot[] valid in thread 0).  Every sum runs in a fixed order, so the result
// is deterministic.
template <int NT, int K, typename A>
__device__ bool ns_reduce(const Prob& pd, State& st, int blk, int nblk, A (&v)[K],
                          double* sh, double* tot) {
  constexpr int NW = NT / 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int is_last;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  // values 0..KS-1 (KS the largest power of two <= min(K, 32)): reduce-scatter
  // across the warp.  At each halving a lane keeps the half of its values
  // selected by its lane bit and adds its partner's copy; then the lane
  // groups' partial sums are added (xor KS .. 16), and lane l < KS ends with
  // value l: KS - 1 + log2(32 / KS) exchanges instead of 5 KS, and one
  // conversion to FP64 per warp instead of KS (FP64 work is slow on this part
  // and queues on one pipe per SM when the CTAs of a launch finish together)
  constexpr int KS = K >= 32 ? 32 : K >= 16 ? 16 : K >= 8 ? 8 : K >= 4 ? 4 : K >= 2 ? 2 : 1;
#pragma unroll
  for (int o = KS / 2; o > 0; o >>= 1) {
    const bool hi = (l & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const A send = hi ? v[i] : v[i + o];
      const A keep = hi ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, o);
    }
  }
#pragma unroll
  for (int o = KS; o < 32; o <<= 1) v[0] += __shfl_xor_sync(FULL, v[0], o);
  if (l < KS) sh[l * NW + w] = (double)v[0];
  constexpr int K0 = KS;
#pragma unroll
  for (int k = K0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
  if (l == 0) {
#pragma unroll
    for (int k = K0; k < K; ++k) sh[k * NW + w] = (double)v[k];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int i = 0; i < NW; ++i) t += sh[threadIdx.x * NW + i];
    pd.partial[(size_t)threadIdx.x * nblk + blk] = t;
    __threadfence();                 // each writer publishes its partial
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(&st.counter, 1u);
    is_last = (prev == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  for (int k = w; k < K; k += NW) {
    // lane l adds blocks l, l + 32, ... in that order; 8 loads in flight at a
    // time (one L2 round trip per 256 blocks rather than per 32)
    const double* pk = pd.partial + (size_t)k * nblk;
    double s = 0.0;
    int i = l;
    for (; i + 7 * 32 < nblk; i += 8 * 32) {
      double a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldcg(pk + i + u * 32);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += a[u];
    }
    for (; i < nblk; i += 32) s += __ldcg(pk + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) tot[k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) st.counter = 0u;
  return true;
}

// root in [0, 1] of the cubic Hermite interpolant with p(0) = h0 < 0 <= p(1)
// = h1 and slopes m0, m1 (per unit t): bisection-safeguarded Newton.  The
// root only seeds the Halley passes (the interpolant itself is off by far
// more than FP32 rounding), so it runs in FP32 to 1e-6 in t: one thread of
// the launch's last block runs it, and a dependent FP64 chain there (long
// FP64 latency on this part) was the longest path of the whole launch.
static __device__ float hermite_root(float h0, float h1, float m0, float m1) {
  auto p = [&](float t, float* dp) {
    const float t2 = t * t, t3 = t2 * t;
    const float H00 = 2.f * t3 - 3.f * t2 + 1.f, H10 = t3 - 2.f * t2 + t;
    const float H01 = -2.f * t3 + 3.f * t2, H11 = t3 - t2;
    *dp = h0 * (6.f * t2 - 6.f * t) + m0 * (3.f * t2 - 4.f * t + 1.f) +
          h1 * (-6.f * t2 + 6.f * t) + m1 * (3.f * t2 - 2.f * t);
    return h0 * H00 + m0 * H10 + h1 * H01 + m1 * H11;
  };
  float lo = 0.f, hi = 1.f;
  float t = (h1 > h0) ? -h0 / (h1 - h0) : 0.5f;
  for (int it = 0; it < 32; ++it) {
    float dp;
    const float v = p(t, &dp);
    if (v < 0.f) lo = t; else hi = t;
    float tn = (dp > 0.f) ? t - v / dp : 0.5f * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
    if (fabsf(tn - t) < 1e-6f || hi - lo < 1e-6f) { t = tn; break; }
    t = tn;
  }
  return t;
}

// Thread 0 of the last block of a bracketing pass: from the totals (h and h'
// sums at the candidates, P last) bracket the root and take the Hermite root.
static __device__ void ns_bracket_finish(const Prob& pd, State& st, const double* tot, double b0) {
  const double P = tot[2 * NS_CAND], target = st.qn * st.qn;
  const double iP = P > 0.0 ? 1.0 / P : 0.0;      // one FP64 division
  auto hv = [&](int j) { return P > 0.0 ? tot[j] * iP - target : 0.0; };
  auto dv = [&](int j) { return 2.0 * tot[NS_CAND + j] * iP; };
  auto bv = [&](int j) { return b0 + (j - 0.5 * (NS_CAND - 1)) * NS_CAND_STEP; };
  int j = 0;
  while (j < NS_CAND && !(hv(j) >= 0.0)) ++j;
  double nb;
  if (j == 0) {
    // root below the window: Newton from the lowest candidate, at most 4 down
    st.nb_lo = -INFINITY; st.nb_hi = bv(0);
    const double d = dv(0);
    nb = (d > 0.0 && isfinite(hv(0) / d)) ? bv(0) - hv(0) / d : bv(0) - 4.0;
    nb = fmax(nb, bv(0) - 4.0);
  } else if (j == NS_CAND) {
    st.nb_lo = bv(NS_CAND - 1); st.nb_hi = INFINITY;
    const double d = dv(NS_CAND - 1);
    nb = (d > 0.0 && isfinite(hv(NS_CAND - 1) / d)) ? bv(NS_CAND - 1) - hv(NS_CAND - 1) / d
                                                    : bv(NS_CAND - 1) + 4.0;
    nb = fmin(nb, bv(NS_CAND - 1) + 4.0);
  } else {
    st.nb_lo = bv(j - 1); st.nb_hi = bv(j);
    const double t = hermite_root((float)hv(j - 1), (float)hv(j), (float)(dv(j - 1) * NS_CAND_STEP),
                                  (float)(dv(j) * NS_CAND_STEP));
    nb = st.nb_lo + t * NS_CAND_STEP;
  }
  st.nphase = 1;
  st.npass += 1;
  ns_set_alpha(pd, st, nb);
}

// accumulate one spectral coefficient (weighted power pf, sigma sf) into the
// candidate sums.  With ci = 1/a_j, x = a_j/(s + a_j) = 1/(1 + s ci) needs one
// FMA and one reciprocal; F_j += pf x^2 and H_j += pf x^3, so that
// G_j = F_j - H_j = sum pf x^2 (1 - x) (the Hermite slopes only seed the
// Halley passes, whose sums form 1 - x directly).  Candidates in pairs:
// two-wide FP32 instructions.
__device__ __forceinline__ void ns_cand_acc(float pf, float sf, const float (&ci)[NS_CAND],
                                            float (&cF)[NS_CAND], float (&cH)[NS_CAND]) {
  const float2 s2 = make_float2(sf, sf), p2 = make_float2(pf, pf), one = make_float2(1.f, 1.f);
#pragma unroll
  for (int j = 0; j < NS_CAND; j += 2) {
    const float2 d = __ffma2_rn(s2, make_float2(ci[j], ci[j + 1]), one);
    const float2 x = make_float2(__fdividef(1.f, d.x), __fdividef(1.f, d.y));
    const float2 px2 = __fmul2_rn(__fmul2_rn(p2, x), x);
    const float2 f = __fadd2_rn(make_float2(cF[j], cF[j + 1]), px2);
    const float2 h = __ffma2_rn(px2, x, make_float2(cH[j], cH[j + 1]));
    cF[j] = f.x; cF[j + 1] = f.y;
    cH[j] = h.x; cH[j + 1] = h.y;
  }
}

// The bracketing pass fused into the forward column pass: the column-pass
// CTA holds its block of the spectrum in shared memory (real view smr:
// transform g's element k at 2 (g TSg + fpad(k)) + {0, 1}), so the candidate
// sums need no second read of S.  DFT: complex column c of the block is
// transform c; DCT: real column c is part (c & 1) of transform c / 2.
template <typename T>
__device__ __noinline__ void ns_cand_block(const Prob& pd, State& st, int blk, const T* smr,
                                           int TSg, size_t base) {
  constexpr int NT = tr_nt(sizeof(T));
  constexpr int K = 2 * NS_CAND + 1;
  __shared__ double red[K * (NT / 32)];
  __shared__ double tot[K];
  __shared__ float s_ci[NS_CAND];
  const int N = pd.n, cb = pd.cb;
  const bool dct = pd.transform == TR_DCT;
  const int W = dct ? N : pd.half;
  const int kb = blk * cb;
  const double b0 = st.nb;
  const T* w = static_cast<const T*>(pd.w) + base;
  T* pwo = static_cast<T*>(pd.pw) + base;   // weighted powers for the Halley passes
  if (threadIdx.x < NS_CAND)
    s_ci[threadIdx.x] = expf(-(float)(b0 + (threadIdx.x - 0.5 * (NS_CAND - 1)) * NS_CAND_STEP));
  __syncthreads();
  float ci[NS_CAND], cF[NS_CAND], cH[NS_CAND];
#pragma unroll
  for (int j = 0; j < NS_CAND; ++j) { ci[j] = s_ci[j]; cF[j] = 0.f; cH[j] = 0.f; }
  const FastDiv fcb(cb);
  T sP = T(0);
  // chunks of MV elements per thread: the chunk's sigma loads first (in
  // flight together), then its sums; a short chunk keeps the unrolled body
  // (MV x NS_CAND = 64 candidate updates) small enough for the instruction cache
  constexpr int MV = 64 / NS_CAND;
#pragma unroll 1
  for (int e0 = 0; e0 < N * cb; e0 += MV * NT) {
  float wv[MV];
#pragma unroll
  for (int qq = 0; qq < MV; ++qq) {
    const int e = e0 + threadIdx.x + qq * NT;
    wv[qq] = (e < N * cb) ? (float)w[e] : 1.f;
  }
#pragma unroll
  for (int qq = 0; qq < MV; ++qq) {
    const int e = e0 + threadIdx.x + qq * NT;
    if (e >= N * cb) break;
    const int k1 = fcb.div(e), c = e - k1 * cb;
    const int k2 = kb + c;
    if (k2 >= W) { pwo[e] = T(0); continue; }
    T pw;
    if (dct) {
      const T v = smr[2 * ((c >> 1) * TSg + fpad(k1)) + (c & 1)];
      pw = T((k1 == 0 ? 1 : 2) * (k2 == 0 ? 1 : 2)) * v * v;
    } else {
      const T vr = smr[2 * (c * TSg + fpad(k1))], vi = smr[2 * (c * TSg + fpad(k1)) + 1];
      const T m = (k2 == 0 || ((N & 1) == 0 && k2 == N / 2)) ? T(1) : T(2);
      pw = m * (vr * vr + vi * vi);
    }
    pwo[e] = pw;
    sP += pw;
    ns_cand_acc((float)pw, wv[qq], ci, cF, cH);
  }
  }
  T v[K];
#pragma unroll
  for (int j = 0; j < NS_CAND; ++j) { v[j] = T(cF[j]); v[NS_CAND + j] = T(cF[j]) - T(cH[j]); }
  v[2 * NS_CAND] = sP;
  if (ns_reduce<NT, K, T>(pd, st, blk, pd.nblk_cols, v, red, tot) && threadIdx.x == 0)
    ns_bracket_finish(pd, st, tot, b0);
}

// four consecutive reals of a row (16-byte aligned for FP32: the row length is
// a multiple of 4 and the buffers are 256-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 u = reinterpret_cast<const double2*>(p)[0], v = reinterpret_cast<const double2*>(p)[1];
  o[0] = u.x; o[1] = u.y; o[2] = v.x; o[3] = v.y;
}
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// two consecutive complex values (one 16-byte access for FP32; p 16-byte aligned)
__device__ __forceinline__ void ldc2(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y); b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ldc2(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }
__device__ __forceinline__ void stc2(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void stc2(double2* p, double2 a, double2 b) { p[0] = a; p[1] = b; }

// ---------------------------------------------------------------------------
// Pass 1: forward transform of row pairs: src (n x n real) -> S
template <typename T>
__device__ __forceinline__ void rows_fwd_body(const int2 item, const Prob* __restrict__ probs, State* __restrict__ states, int src_slot, int pcg) {
  using T2 = typename Vec2<T>::type;
  constexpr int NT = tr_nt(sizeof(T)), MAXV = TR_CAP / NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const Prob& pd = probs[item.x];
  if (tr_skip(states[pd.sidx], pcg)) return;
  const int N = pd.n, G = pd.row_g, TSg = fpad(N) + 1;
  const int pair0 = item.y * G;
  const int row0 = 2 * pair0;
  const bool dct = (pd.transform == TR_DCT);
  const T* src = static_cast<const T*>(pd.buf[src_slot]);
  const FastDiv fN(N);
  if ((N & 3) == 0) {
    // rows in groups of 4 reals, one vector load per group and row; sample
    // y = 4 xq + i goes to position y (DFT) or to its DCT position (even y to
    // y / 2, odd y to N - 1 - (y - 1) / 2).  All loads first, then the stores.
    constexpr int MQ = MAXV / 4;
    const int NQ = N >> 2;
    const FastDiv fq(NQ);
    T a[MQ][4], b[MQ][4];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e < G * NQ) {
        const int g = fq.div(e), xq = e - g * NQ;
        const int ra = row0 + 2 * g;
        const T* r = src + (size_t)ra * N + 4 * xq;
        if (ra < N) ld4(r, a[q]); else a[q][0] = a[q][1] = a[q][2] = a[q][3] = T(0);
        if (ra + 1 < N) ld4(r + N, b[q]); else b[q][0] = b[q][1] = b[q][2] = b[q][3] = T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e < G * NQ) {
        const int g = fq.div(e), xq = e - g * NQ;
        T2* tb = sm + g * TSg;
        const int p0 = dct ? 2 * xq : 4 * xq, p1 = dct ? N - 1 - 2 * xq : 4 * xq + 1;
        const int p2 = dct ? 2 * xq + 1 : 4 * xq + 2, p3 = dct ? N - 2 - 2 * xq : 4 * xq + 3;
        tb[fpad(p0)] = mk2<T2>(a[q][0], b[q][0]);
        tb[fpad(p1)] = mk2<T2>(a[q][1], b[q][1]);
        tb[fpad(p2)] = mk2<T2>(a[q][2], b[q][2]);
        tb[fpad(p3)] = mk2<T2>(a[q][3], b[q][3]);
      }
    }
  } else {
    // all loads of this thread first (up to MAXV in flight), then the stores
    T2 tmp[MAXV];
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e < G * N) {
        const int g = fN.div(e), x = e - g * N;
        const int ra = row0 + 2 * g, rb = ra + 1;
        const int xs = dct ? dct_src(x, N) : x;
        tmp[q].x = (ra < N) ? src[(size_t)ra * N + xs] : T(0);
        tmp[q].y = (rb < N) ? src[(size_t)rb * N + xs] : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      const int e = threadIdx.x + q * NT;
      if (e < G * N) { const int g = fN.div(e), x = e - g * N; sm[g * TSg + fpad(x)] = tmp[q]; }
    }
  }
  __syncthreads();
  fft_smem<T2, false>(G, pd);
  if (dct) dct_split<T, T2>(sm, G, N, TSg, static_cast<const T2*>(pd.dtw));
  // write the rows of this CTA into every column block (contiguous runs)
  const int W = dct ? N : pd.half;
  const int cb = pd.cb;
  const int R2 = 2 * G;
  const int nb = (W + cb - 1) / cb;
  // spectral value k of local row rl
  auto spec_val = [&](const T2* tb, int rl, int k) -> T2 {
    if (dct) {
      const T2 X = tb[fpad(k)];
      T2 r; r.x = (rl & 1) ? X.y : X.x; r.y = T(0); return r;
    }
    const T2 Z = tb[fpad(k)];
    const T2 Zr = tb[fpad(k == 0 ? 0 : N - k)];
    T2 X;
    if (rl & 1) { X.x = T(0.5) * (Z.y + Zr.y); X.y = T(-0.5) * (Z.x - Zr.x); }   // (Z - conj Zr)/(2i)
    else { X.x = T(0.5) * (Z.x + Zr.x); X.y = T(0.5) * (Z.y - Zr.y); }           // (Z + conj Zr)/2
    return X;
  };
  if ((cb & 1) == 0) {
    // columns in pairs (c, c + 1): one 8-byte (DCT) or 16-byte (DFT) store
    const int H = cb / 2;
    const FastDiv frh(R2 * H), fh(H);
    for (int e = threadIdx.x; e < nb * R2 * H; e += NT) {
      const int b = frh.div(e), rem = e - b * (R2 * H);
      const int rl = fh.div(rem), c = 2 * (rem - rl * H);
      const int k = b * cb + c, row = row0 + rl;
      if (k >= W || row >= N) continue;
      const T2* tb = sm + (rl >> 1) * TSg;
      const size_t o = (size_t)b * N * cb + (size_t)row * cb + c;
      const bool two = k + 1 < W;
      const T2 x0 = spec_val(tb, rl, k);
      if (dct) {
        T* S = static_cast<T*>(pd.buf[SL_S]);
        if (two) *reinterpret_cast<T2*>(S + o) = mk2<T2>(x0.x, spec_val(tb, rl, k + 1).x);
        else S[o] = x0.x;
      } else {
        T2* S = static_cast<T2*>(pd.buf[SL_S]);
        if (two) stc2(S + o, x0, spec_val(tb, rl, k + 1));
        else S[o] = x0;
      }
    }
    return;
  }
  const FastDiv frc(R2 * cb), fcb(cb);
  for (int e = threadIdx.x; e < nb * R2 * cb; e += NT) {
    const int b = frc.div(e), rem = e - b * (R2 * cb);
    const int rl = fcb.div(rem), c = rem - rl * cb;
    const int k = b * cb + c, row = row0 + rl;
    if (k >= W || row >= N) continue;
    const T2* tb = sm + (rl >> 1) * TSg;
    const size_t o = (size_t)b * N * cb + (size_t)row * cb + c;
    if (dct) {
      const T2 X = tb[fpad(k)];
      static_cast<T*>(pd.buf[SL_S])[o] = (rl & 1) ? X.y : X.x;
    } else {
      const T2 Z = tb[fpad(k)];
      const T2 Zr = tb[fpad(k == 0 ? 0 : N - k)];
      T2 X;
      if (rl & 1) { X.x = T(0.5) * (Z.y + Zr.y); X.y = T(-0.5) * (Z.x - Zr.x); }   // (Z - conj Zr)/(2i)
      else { X.x = T(0.5) * (Z.x + Zr.x); X.y = T(0.5) * (Z.y - Zr.y); }           // (Z + conj Zr)/2
      static_cast<T2*>(pd.buf[SL_S])[o] = X;
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(tr_nt(sizeof(T)), tr_minb(sizeof(T)))
k_rows_fwd(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items, int src_slot, int pcg) {
  rows_fwd_body<T>(items[blockIdx.x], probs, states, src_slot, pcg);
}


// spectral weight at blocked index idx; alpha and kind as given.  |lambda|^2 +
// alpha is formed in T: alpha > 0 keeps it away from zero (no cancellation),
// so FP32 holds it to 6e-8 relative; 1/n^2 of the unnormalised pair is folded in.
// scale / (|lambda|^2 + alpha): the fast reciprocal-based quotient in FP32
// (within 2 ulp), the exact one in FP64
__device__ __forceinline__ float wdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double wdiv(double a, double b) { return a / b; }

template <typename T, typename T2>
__device__ __forceinline__ T2 weight_dft(const Prob& pd, size_t idx, T alpha, T scale, int kind) {
  const T inv = wdiv(scale, static_cast<const T*>(pd.w)[idx] + alpha);
  T2 w;
  if (kind == W_TIKH) {
    const T2 l = static_cast<const T2*>(pd.lam)[idx];
    w.x = l.x * inv; w.y = -l.y * inv;
  } else { w.x = inv; w.y = T(0); }
  return w;
}
template <typename T>
__device__ __forceinline__ T weight_dct(const Prob& pd, size_t idx, T alpha, T scale, int kind) {
  const T inv = wdiv(scale, static_cast<const T*>(pd.w)[idx] + alpha);
  return kind == W_TIKH ? static_cast<const T*>(pd.lam)[idx] * inv : inv;
}
// the weights of real columns idx and idx + 1 (idx even: one aligned pair load)
template <typename T, typename T2>
__device__ __forceinline__ T2 weight_dct2(const Prob& pd, size_t idx, T alpha, T scale, int kind) {
  const T2 s = *reinterpret_cast<const T2*>(static_cast<const T*>(pd.w) + idx);
  T2 r;
  r.x = wdiv(scale, s.x + alpha);
  r.y = wdiv(scale, s.y + alpha);
  if (kind == W_TIKH) {
    const T2 l = *reinterpret_cast<const T2*>(static_cast<const T*>(pd.lam) + idx);
    r.x *= l.x; r.y *= l.y;
  }
  return r;
}

// Pass 2: one column block per CTA.  DFT: cb complex columns; DCT: cb real
// columns = cb/2 packed pairs.
// (the mode is a template parameter: each launch runs only its own code; the
// two 4-NS modes measured faster at 5 FP32 CTAs per SM, the others at 4)
template <typename T, int mode>
__device__ __forceinline__ void cols_body(const int2 item, const Prob* __restrict__ probs,
                                          State* __restrict__ states, int pcg, double op_alpha,
                                          int op_kind) {
  using T2 = typename Vec2<T>::type;
  constexpr int NT = tr_nt(sizeof(T)), MAXV = TR_CAP / NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const Prob& pd = probs[item.x];
  State& st = states[pd.sidx];
  if (tr_skip(st, pcg)) return;
  // Algorithm 4-NS past the discrepancy point keeps alpha_n (no solve this
  // iteration): the forward pass then weights and inverts at once, as the
  // stationary pass does, and the inverse pass has nothing left to do
  const bool kept = mode == COL_FWD && !pcg && pd.ns && !st.ns_active;
  if (mode == COL_NS_INV && (!pd.ns || !st.ns_active)) return;
  // Algorithm 4-NS: the forward pass also runs the bracketing pass of alpha_n
  const bool cand = mode == COL_FWD && !pcg && pd.ns && st.ns_active && !st.nconv && st.nphase == 0;
  const int N = pd.n, cb = pd.cb, TSg = fpad(N) + 1;
  const bool dct = (pd.transform == TR_DCT);
  // weight parameters
  double alpha = pd.alpha;
  int kind = (pd.precond == P_TIKH || pd.precond == P_TIKH_NS) && pd.bc != BC_RECT ? W_TIKH : W_INV;
  if (mode == COL_NS_INV || kept) alpha = st.alpha_n;
  if (mode == COL_OP) { alpha = op_alpha; kind = op_kind; }
  if (pd.precond == P_KRYLOV) kind = W_INV;
  const T Ta = T(alpha);
  // 1/n^2 (n^2 < 2^24 is exact in FP32; the FP64 division stays in FP64 runs)
  const T Tsc = T(1) / T((double)pd.n * (double)pd.n);
  const size_t base = (size_t)item.y * N * cb;       // this CTA's contiguous block
  const int W = dct ? N : pd.half;
  const int kb = item.y * cb;                         // first column of the block
  // The weights |lambda|^2 (and lambda) of this block are read only after the
  // forward transform (|lambda|^2 also by the bracketing pass); ask L2 for
  // their lines now so that the HBM latency overlaps the block load and the
  // passes (one prefetch per 128-byte line)
  if (mode != COL_FWD || kept || cand) {
    const char* ws = reinterpret_cast<const char*>(static_cast<const T*>(pd.w) + base);
    const size_t wb = (size_t)N * cb * sizeof(T);
    for (size_t o = (size_t)threadIdx.x * 128; o < wb; o += (size_t)NT * 128) prefetch_l2(ws + o);
    if (kind == W_TIKH && !cand) {
      const size_t le = dct ? sizeof(T) : 2 * sizeof(T);
      const char* ls = static_cast<const char*>(pd.lam) + base * le;
      for (size_t o = (size_t)threadIdx.x * 128; o < (size_t)N * cb * le; o += (size_t)NT * 128)
        prefetch_l2(ls + o);
    }
  }
  if (!dct && (cb & 1) == 0) {
    // an even number of complex columns: columns 2h and 2h + 1 (transforms
    // 2h, 2h + 1) move together, quad (k1, h) at 2 (k1 cb / 2 + h)
    const int G = cb, H = cb / 2;
    const FastDiv fH(H);
    T2* S = static_cast<T2*>(pd.buf[SL_S]) + base;
    const int NQ = N * H;
    const int nvc = W - kb < cb ? W - kb : cb;      // valid columns of the block
    {
      T2 ta[MAXV / 2], tb[MAXV / 2];
#pragma unroll
      for (int q = 0; q < MAXV / 2; ++q) {
        const int e = threadIdx.x + q * NT;
        ta[q].x = ta[q].y = tb[q].x = tb[q].y = T(0);
        if (e < NQ) {
          const int c = 2 * (e - fH.div(e) * H);
          if (c + 1 < nvc) ldc2(S + 2 * e, ta[q], tb[q]);
          else if (c < nvc) ta[q] = S[2 * e];
        }
      }
#pragma unroll
      for (int q = 0; q < MAXV / 2; ++q) {
        const int e = threadIdx.x + q * NT;
        if (e < NQ) {
          const int k1 = fH.div(e), c = 2 * (e - k1 * H);
          T2 a = ta[q], b = tb[q];
          if (mode == COL_NS_INV) {
            // no forward transform: the weights are applied on the way in
            if (c < nvc) a = cmul(a, weight_dft<T, T2>(pd, base + 2 * (size_t)e, Ta, Tsc, kind));
            if (c + 1 < nvc) b = cmul(b, weight_dft<T, T2>(pd, base + 2 * (size_t)e + 1, Ta, Tsc, kind));
          }
          sm[c * TSg + fpad(k1)] = a;
          sm[(c + 1) * TSg + fpad(k1)] = b;
        }
      }
    }
    __syncthreads();
    auto put = [&](int e, int k1, int c) {
      const T2 a = sm[c * TSg + fpad(k1)], b = sm[(c + 1) * TSg + fpad(k1)];
      if (c + 1 < nvc) stc2(S + 2 * e, a, b);
      else if (c < nvc) S[2 * e] = a;
    };
    if (mode != COL_NS_INV) fft_smem<T2, false>(G, pd);
    if (mode == COL_FWD && !kept) {
      for (int e = threadIdx.x; e < NQ; e += NT) {
        const int k1 = fH.div(e), c = 2 * (e - k1 * H);
        put(e, k1, c);
      }
      if (cand) ns_cand_block<T>(pd, st, item.y, reinterpret_cast<const T*>(sm), TSg, base);
      return;
    }
    if (mode != COL_NS_INV) {
      for (int e = threadIdx.x; e < NQ; e += NT) {
        const int k1 = fH.div(e), c = 2 * (e - k1 * H);
        if (c < nvc) {
          T2& v = sm[c * TSg + fpad(k1)];
          v = cmul(v, weight_dft<T, T2>(pd, base + 2 * (size_t)e, Ta, Tsc, kind));
        }
        if (c + 1 < nvc) {
          T2& v = sm[(c + 1) * TSg + fpad(k1)];
          v = cmul(v, weight_dft<T, T2>(pd, base + 2 * (size_t)e + 1, Ta, Tsc, kind));
        }
      }
      __syncthreads();
    }
    fft_smem<T2, true>(G, pd);
    for (int e = threadIdx.x; e < NQ; e += NT) {
      const int k1 = fH.div(e), c = 2 * (e - k1 * H);
      put(e, k1, c);
    }
  } else if (!dct) {
    const int G = cb;
    const FastDiv fG(G);
    T2* S = static_cast<T2*>(pd.buf[SL_S]) + base;
    {
      T2 tmp[MAXV];
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        const int e = threadIdx.x + q * NT;
        tmp[q].x = T(0); tmp[q].y = T(0);
        if (e < N * G && kb + (e - fG.div(e) * G) < W) tmp[q] = S[e];
      }
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        const int e = threadIdx.x + q * NT;
        if (e < N * G) { const int k1 = fG.div(e), c = e - k1 * G; sm[c * TSg + fpad(k1)] = tmp[q]; }
      }
    }
    __syncthreads();
    if (mode != COL_NS_INV) fft_smem<T2, false>(G, pd);
    if (mode == COL_FWD && !kept) {
      for (int e = threadIdx.x; e < N * G; e += NT) {
        const int k1 = fG.div(e), c = e - k1 * G;
        if (kb + c < W) S[e] = sm[c * TSg + fpad(k1)];
      }
      if (cand) ns_cand_block<T>(pd, st, item.y, reinterpret_cast<const T*>(sm), TSg, base);
      return;
    }
    for (int e = threadIdx.x; e < N * G; e += NT) {
      const int k1 = fG.div(e), c = e - k1 * G;
      if (kb + c < W) {
        T2& v = sm[c * TSg + fpad(k1)];
        v = cmul(v, weight_dft<T, T2>(pd, base + e, Ta, Tsc, kind));
      }
    }
    __syncthreads();
    fft_smem<T2, true>(G, pd);
    for (int e = threadIdx.x; e < N * G; e += NT) {
      const int k1 = fG.div(e), c = e - k1 * G;
      if (kb + c < W) S[e] = sm[c * TSg + fpad(k1)];
    }
  } else {
    // real columns 2g and 2g + 1 of the block are transform g (real and
    // imaginary part): the block moves as N G pairs, pair (k1, g) at 2 (k1 G + g)
    const int G = cb / 2;
    const FastDiv fG(G);
    T* S = static_cast<T*>(pd.buf[SL_S]) + base;
    T2* S2 = reinterpret_cast<T2*>(S);          // cb even, base even: aligned pairs
    T* smr = reinterpret_cast<T*>(sm);
    const int NP = N * G;
    // valid real columns of this block (the last block may be padded)
    const int nvc = W - kb < cb ? W - kb : cb;
    {
      T2 tmp[MAXV];
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        const int e = threadIdx.x + q * NT;
        tmp[q].x = T(0); tmp[q].y = T(0);
        if (e < NP) {
          const int c = 2 * (e - fG.div(e) * G);
          if (c + 1 < nvc) tmp[q] = S2[e];
          else if (c < nvc) tmp[q].x = S[2 * e];
        }
      }
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        const int e = threadIdx.x + q * NT;
        if (e < NP) {
          const int k1 = fG.div(e), g = e - k1 * G;
          const int pos = (mode == COL_NS_INV) ? k1 : dct_pos(k1, N);
          T2 v = tmp[q];
          if (mode == COL_NS_INV) {
            // no forward transform: the weights are applied on the way in
            const int c = 2 * g;
            if (c + 1 < nvc) {
              const T2 w = weight_dct2<T, T2>(pd, base + 2 * (size_t)e, Ta, Tsc, kind);
              v.x *= w.x; v.y *= w.y;
            } else if (c < nvc) {
              v.x *= weight_dct<T>(pd, base + 2 * (size_t)e, Ta, Tsc, kind);
            }
          }
          sm[g * TSg + fpad(pos)] = v;
        }
      }
    }
    __syncthreads();
    const T2* dtw = static_cast<const T2*>(pd.dtw);
    if (mode != COL_NS_INV) {
      fft_smem<T2, false>(G, pd);
      dct_split<T, T2>(sm, G, N, TSg, dtw);
    }
    // store pair e from shared-memory position pos of its transform
    auto put = [&](int e, int g, int pos) {
      const int c = 2 * g;
      const T2 v = sm[g * TSg + fpad(pos)];
      if (c + 1 < nvc) S2[e] = v;
      else if (c < nvc) S[2 * e] = v.x;
    };
    if (mode == COL_FWD && !kept) {
      for (int e = threadIdx.x; e < NP; e += NT) {
        const int k1 = fG.div(e), g = e - k1 * G;
        put(e, g, k1);
      }
      if (cand) ns_cand_block<T>(pd, st, item.y, smr, TSg, base);
      return;
    }
    if (mode != COL_NS_INV) {
      for (int e = threadIdx.x; e < NP; e += NT) {
        const int k1 = fG.div(e), g = e - k1 * G;
        const int c = 2 * g;
        T2& v = sm[g * TSg + fpad(k1)];
        if (c + 1 < nvc) {
          const T2 w = weight_dct2<T, T2>(pd, base + 2 * (size_t)e, Ta, Tsc, kind);
          v.x *= w.x; v.y *= w.y;
        } else {
          v.x *= (c < nvc) ? weight_dct<T>(pd, base + 2 * (size_t)e, Ta, Tsc, kind) : T(0);
          v.y = T(0);
        }
      }
      __syncthreads();
    }
    dct_merge<T, T2>(sm, G, N, TSg, dtw);
    fft_smem<T2, true>(G, pd);
    for (int e = threadIdx.x; e < NP; e += NT) {
      const int k1 = fG.div(e), g = e - k1 * G;
      put(e, g, dct_pos(k1, N));
    }
  }
}
template <typename T, int mode>
__global__ void __launch_bounds__(tr_nt(sizeof(T)),
                                  tr_minb(sizeof(T)) + ((sizeof(T) == 4 && (mode == COL_FWD || mode == COL_NS_INV)) ? 1 : 0))
k_cols(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
       int pcg, double op_alpha, int op_kind) {
  cols_body<T, mode>(items[blockIdx.x], probs, states, pcg, op_alpha, op_kind);
}

// Pass 3: inverse transform of row pairs: S -> dst (n x n real)
template <typename T>
__device__ __forceinline__ void rows_inv_body(const int2 item, const Prob* __restrict__ probs, State* __restrict__ states, int dst_slot, int pcg) {
  using T2 = typename Vec2<T>::type;
  constexpr int NT = tr_nt(sizeof(T));
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const Prob& pd = probs[item.x];
  if (tr_skip(states[pd.sidx], pcg)) return;
  const int N = pd.n, G = pd.row_g, TSg = fpad(N) + 1;
  const int row0 = 2 * item.y * G;
  const bool dct = (pd.transform == TR_DCT);
  // Loads walk the column blocks: within block b the 2G rows of this CTA are
  // one contiguous run of 2G cb elements; thread e takes column c of pair g.
  const int cb = pd.cb;
  const int W = dct ? N : pd.half;
  const int nb = (W + cb - 1) / cb;
  const int tot = nb * G * cb;
  const FastDiv fgc(G * cb), fcb(cb), fN(N);
  constexpr int BATCH = 8;
  const bool even = (N & 1) == 0;
  // Z[k] = Xa[k] + i Xb[k] of the DFT rows (the missing half from Hermitian
  // symmetry), or the packed pair (Xa, Xb) of the DCT rows, into transform g
  auto put_dft = [&](T2* tb, int kk, T2 xa, T2 xb) {
    if (kk == 0 || (even && kk == N / 2)) {
      T2 z; z.x = xa.x; z.y = xb.x;        // imaginary parts of DC / Nyquist are rounding
      tb[fpad(kk)] = z;
    } else {
      T2 z; z.x = xa.x - xb.y; z.y = xa.y + xb.x;     // Xa + i Xb
      tb[fpad(kk)] = z;
      T2 zr; zr.x = xa.x + xb.y; zr.y = xb.x - xa.y;  // conj(Xa) + i conj(Xb)
      tb[fpad(N - kk)] = zr;
    }
  };
  if ((cb & 1) == 0) {
    // columns in pairs (c, c + 1): one 8-byte (DCT) or 16-byte (DFT) load per
    // row of the pair
    constexpr int BATCH2 = 4;          // 4 pairs of 2 rows x 2 columns in flight
    const int H = cb / 2;
    const int tot2 = nb * G * H;
    const FastDiv fgh(G * H), fh(H);
    for (int e0 = threadIdx.x; e0 < tot2; e0 += BATCH2 * NT) {
      T2 a0[BATCH2], a1[BATCH2], b0[BATCH2], b1[BATCH2];
      int kq[BATCH2];
#pragma unroll
      for (int u = 0; u < BATCH2; ++u) {
        const int e = e0 + u * NT;
        kq[u] = -1;
        a0[u].x = a0[u].y = a1[u].x = a1[u].y = T(0);
        b0[u] = a0[u]; b1[u] = a0[u];
        if (e < tot2) {
          const int b = fgh.div(e), rem = e - b * (G * H);
          const int g = fh.div(rem), c = 2 * (rem - g * H);
          const int ra = row0 + 2 * g;
          const int k = b * cb + c;
          if (k < W) {
            const size_t o = (size_t)b * N * cb + (size_t)ra * cb + c;
            if (dct) {
              const T* S = static_cast<const T*>(pd.buf[SL_S]);
              if (ra < N) a0[u] = *reinterpret_cast<const T2*>(S + o);        // row ra, columns c, c + 1
              if (ra + 1 < N) b0[u] = *reinterpret_cast<const T2*>(S + o + cb);
            } else {
              const T2* S = static_cast<const T2*>(pd.buf[SL_S]);
              if (ra < N) ldc2(S + o, a0[u], a1[u]);
              if (ra + 1 < N) ldc2(S + o + cb, b0[u], b1[u]);
            }
            kq[u] = (g << 16) | k;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < BATCH2; ++u) {
        if (kq[u] < 0) continue;
        const int k = kq[u] & 0xffff;
        T2* tb = sm + (kq[u] >> 16) * TSg;
        const bool two = k + 1 < W;
        if (dct) {
          tb[fpad(k)] = mk2<T2>(a0[u].x, b0[u].x);
          if (two) tb[fpad(k + 1)] = mk2<T2>(a0[u].y, b0[u].y);
        } else {
          put_dft(tb, k, a0[u], b0[u]);
          if (two) put_dft(tb, k + 1, a1[u], b1[u]);
        }
      }
    }
    __syncthreads();
    if (dct) dct_merge<T, T2>(sm, G, N, TSg, static_cast<const T2*>(pd.dtw));
  } else if (dct) {
    const T* S = static_cast<const T*>(pd.buf[SL_S]);
    for (int e0 = threadIdx.x; e0 < tot; e0 += BATCH * NT) {
      T2 v[BATCH];
      int k[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = e0 + u * NT;
        k[u] = -1;
        if (e < tot) {
          const int b = fgc.div(e), rem = e - b * (G * cb);
          const int g = fcb.div(rem), c = rem - g * cb;
          const int ra = row0 + 2 * g;
          const size_t o = (size_t)b * N * cb + (size_t)ra * cb + c;
          k[u] = b * cb + c;
          v[u].x = (ra < N && k[u] < W) ? S[o] : T(0);
          v[u].y = (ra + 1 < N && k[u] < W) ? S[o + cb] : T(0);
          k[u] = (k[u] < W) ? (g << 16) | k[u] : -1;
        }
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u)
        if (k[u] >= 0) sm[(k[u] >> 16) * TSg + fpad(k[u] & 0xffff)] = v[u];
    }
    __syncthreads();
    dct_merge<T, T2>(sm, G, N, TSg, static_cast<const T2*>(pd.dtw));
  } else {
    // Z[k] = Xa[k] + i Xb[k]; the missing half from Hermitian symmetry
    const bool even = (N & 1) == 0;
    const T2* S = static_cast<const T2*>(pd.buf[SL_S]);
    for (int e0 = threadIdx.x; e0 < tot; e0 += BATCH * NT) {
      T2 xa[BATCH], xb[BATCH];
      int k[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = e0 + u * NT;
        k[u] = -1;
        xa[u].x = xa[u].y = xb[u].x = xb[u].y = T(0);
        if (e < tot) {
          const int b = fgc.div(e), rem = e - b * (G * cb);
          const int g = fcb.div(rem), c = rem - g * cb;
          const int ra = row0 + 2 * g;
          const int kk = b * cb + c;
          if (kk < W) {
            const size_t o = (size_t)b * N * cb + (size_t)ra * cb + c;
            if (ra < N) xa[u] = S[o];
            if (ra + 1 < N) xb[u] = S[o + cb];
            k[u] = (g << 16) | kk;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        if (k[u] < 0) continue;
        const int kk = k[u] & 0xffff;
        T2* tb = sm + (k[u] >> 16) * TSg;
        if (kk == 0 || (even && kk == N / 2)) {
          T2 z; z.x = xa[u].x; z.y = xb[u].x;        // imaginary parts of DC / Nyquist are rounding
          tb[fpad(kk)] = z;
        } else {
          T2 z; z.x = xa[u].x - xb[u].y; z.y = xa[u].y + xb[u].x;     // Xa + i Xb
          tb[fpad(kk)] = z;
          T2 zr; zr.x = xa[u].x + xb[u].y; zr.y = xb[u].x - xa[u].y;  // conj(Xa) + i conj(Xb)
          tb[fpad(N - kk)] = zr;
        }
      }
    }
    __syncthreads();
  }
  fft_smem<T2, true>(G, pd);
  T* dst = static_cast<T*>(pd.buf[dst_slot]);
  if ((N & 3) == 0) {
    // groups of 4 reals per row, one vector store per group and row
    const int NQ = N >> 2;
    const FastDiv fq(NQ);
    for (int e = threadIdx.x; e < G * NQ; e += NT) {
      const int g = fq.div(e), xq = e - g * NQ;
      const int ra = row0 + 2 * g;
      const T2* tb = sm + g * TSg;
      const int p0 = dct ? 2 * xq : 4 * xq, p1 = dct ? N - 1 - 2 * xq : 4 * xq + 1;
      const int p2 = dct ? 2 * xq + 1 : 4 * xq + 2, p3 = dct ? N - 2 - 2 * xq : 4 * xq + 3;
      const T2 v0 = tb[fpad(p0)], v1 = tb[fpad(p1)], v2 = tb[fpad(p2)], v3 = tb[fpad(p3)];
      T* r = dst + (size_t)ra * N + 4 * xq;
      if (ra < N) st4(r, v0.x, v1.x, v2.x, v3.x);
      if (ra + 1 < N) st4(r + N, v0.y, v1.y, v2.y, v3.y);
    }
    return;
  }
  for (int e = threadIdx.x; e < G * N; e += NT) {
    const int g = fN.div(e), x = e - g * N;
    const int ra = row0 + 2 * g, rb = ra + 1;
    const T2 v = sm[g * TSg + fpad(dct ? dct_pos(x, N) : x)];
    if (ra < N) dst[(size_t)ra * N + x] = v.x;
    if (rb < N) dst[(size_t)rb * N + x] = v.y;
  }
}
template <typename T>
__global__ void __launch_bounds__(tr_nt(sizeof(T)), tr_minb(sizeof(T)))
k_rows_inv(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items, int dst_slot, int pcg) {
  rows_inv_body<T>(items[blockIdx.x], probs, states, dst_slot, pcg);
}


// Bracketing pass (nphase 0): h and h' at NS_CAND candidates around the
// previous root.
template <typename T>
__global__ void __launch_bounds__(NS_NT, 2)
k_spec_cand(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items) {
  constexpr int K = 2 * NS_CAND + 1;
  __shared__ double red[K * (NS_NT / 32)];
  __shared__ double tot[K];
  __shared__ float s_ci[NS_CAND];
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  State& st = states[item.x];
  if (st.stopped || !pd.ns || !st.ns_active || st.nconv || st.nphase != 0) return;
  const double b0 = st.nb;
  if (threadIdx.x < NS_CAND)
    s_ci[threadIdx.x] = expf(-(float)(b0 + (threadIdx.x - 0.5 * (NS_CAND - 1)) * NS_CAND_STEP));
  __syncthreads();
  float ci[NS_CAND], cF[NS_CAND], cH[NS_CAND];
#pragma unroll
  for (int j = 0; j < NS_CAND; ++j) { ci[j] = s_ci[j]; cF[j] = 0.f; cH[j] = 0.f; }
  T sP = T(0);
#pragma unroll 1
  for (int q0 = 0; q0 < NS_PT; q0 += NS_B) {
    T pw[NS_B], sg[NS_B];
    bool ok[NS_B];
#pragma unroll
    for (int q = 0; q < NS_B; ++q)
      ok[q] = spec_elem<T>(pd, item.y, threadIdx.x + (q0 + q) * NS_NT, pw[q], sg[q]);
#pragma unroll
    for (int q = 0; q < NS_B; ++q) {
      const int L = item.y * (NS_NT * NS_PT) + threadIdx.x + (q0 + q) * NS_NT;
      if (L < pd.nblk_cols * pd.n * pd.cb) static_cast<T*>(pd.pw)[L] = ok[q] ? pw[q] : T(0);
      if (!ok[q]) continue;
      sP += pw[q];
      ns_cand_acc((float)pw[q], (float)sg[q], ci, cF, cH);
    }
  }
  T v[K];
#pragma unroll
  for (int j = 0; j < NS_CAND; ++j) { v[j] = T(cF[j]); v[NS_CAND + j] = T(cF[j]) - T(cH[j]); }
  v[2 * NS_CAND] = sP;
  if (ns_reduce<NS_NT, K, T>(pd, st, item.y, pd.nblk_spec, v, red, tot) && threadIdx.x == 0)
    ns_bracket_finish(pd, st, tot, b0);
}

// Refinement pass (nphase 1): a safeguarded Halley step at the current b.
template <typename T>
__device__ __forceinline__ void spec_body(const int2 item, const Prob* __restrict__ probs, State* __restrict__ states) {
  __shared__ double red[4 * (NS_NT / 32)];
  __shared__ double tot[4];
  const Prob& pd = probs[item.x];
  State& st = states[item.x];
  if (st.stopped || !pd.ns || !st.ns_active || st.nconv || st.nphase != 1) return;
  const double b0 = st.nb;
  // exp(b0), formed in FP64 where b0 was set (FP64 latency is long on this
  // part: no exp per CTA)
  const T alpha = T(st.ea);
  // the weighted powers (0 on padding) and sigma, both blocked like S
  const int nel = pd.nblk_cols * pd.n * pd.cb;
  const T* P = static_cast<const T*>(pd.pw);
  const T* Sg = static_cast<const T*>(pd.w);
  int L = item.y * (NS_NT * NS_PT) + threadIdx.x;
  T sP = T(0), sF = T(0), sG1 = T(0), sG2 = T(0);
#pragma unroll 1
  for (int q0 = 0; q0 < NS_PT; q0 += NS_B) {
    T pw[NS_B], sg[NS_B];
#pragma unroll
    for (int q = 0; q < NS_B; ++q) {
      const int e = L + q * NS_NT;
      pw[q] = T(0); sg[q] = T(1);
      if (e < nel) { pw[q] = P[e]; sg[q] = Sg[e]; }
    }
#pragma unroll
    for (int q = 0; q < NS_B; ++q) {
      const T x = wdiv(alpha, sg[q] + alpha);
      const T px2 = pw[q] * x * x;
      const T g1 = px2 * (T(1) - x);
      sP += pw[q];
      sF += px2;
      sG1 += g1;
      sG2 += g1 * (T(2) - T(3) * x);
    }
    L += NS_B * NS_NT;
  }
  T v[4] = {sP, sF, sG1, sG2};
  if (ns_reduce<NS_NT, 4, T>(pd, st, item.y, pd.nblk_spec, v, red, tot) && threadIdx.x == 0) {
    const double P = tot[0];
    const double target = st.qn * st.qn;
    const double iP = (P > 0.0) ? 1.0 / P : 0.0;  // one FP64 division
    const double h = (P > 0.0) ? tot[1] * iP - target : 0.0;
    const double h1 = 2.0 * tot[2] * iP;
    const double h2 = 2.0 * tot[3] * iP;
    const double nb = b0;
    if (h < 0.0) st.nb_lo = fmax(st.nb_lo, nb);
    else if (h > 0.0) st.nb_hi = fmin(st.nb_hi, nb);
    double step = 0.0;
    bool have = false;
    if (h1 > 0.0) {
      const double den = 2.0 * h1 * h1 - h * h2;
      step = (den > 0.0) ? 2.0 * h * h1 / den : h / h1;     // Halley, else Newton
      have = isfinite(step);
    }
    double nn = have ? nb - step : ((h < 0.0) ? nb + 2.0 : nb - 2.0);
    const bool inside = nn >= st.nb_lo && nn <= st.nb_hi;
    bool conv = have && inside &&
                (fabs(step) <= ns_tol(sizeof(T)) || fabs(step) <= ns_tol3(sizeof(T)));
    if (!conv) {
      if (isfinite(st.nb_lo) && isfinite(st.nb_hi)) {
        if (!inside) nn = 0.5 * (st.nb_lo + st.nb_hi);
      } else {
        if (nn > nb + 4.0) nn = nb + 4.0;
        if (nn < nb - 4.0) nn = nb - 4.0;
      }
    }
    st.npass += 1;
    if (conv || st.npass >= 40) st.nconv = 1;
    ns_set_alpha(pd, st, nn);
  }
}
template <typename T>
__global__ void __launch_bounds__(NS_NT)
k_spec(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items) {
  spec_body<T>(items[blockIdx.x], probs, states);
}



// ---------------------------------------------------------------------------
// The antireflective transform (Section 2.2), for antireflective BCs with a
// quadrantally symmetric PSF:
//   T = [ 1 - i/(n-1) | sin(j pi i/(n-1)), j = 1..n-2 | i/(n-1) ],
//   T^{-1} x: c_0 = x_0, c_{n-1} = x_{n-1},
//             c_j = (2/(n-1)) sum_i sin(j pi i/(n-1)) (x_i - x_0 (1 - t_i) - x_{n-1} t_i)
//   T c:      x_0 = c_0, x_{n-1} = c_{n-1},
//             x_i = sum_j sin(j pi i/(n-1)) c_j + c_0 (1 - t_i) + c_{n-1} t_i,
// t_i = i/(n-1), i, j = 1..n-2.  The sine sums (a DST-I of length n - 2) are
// one DFT of length M = 2(n-1) (pd.nfft) of the odd extension
// (0, y_1 .. y_{n-2}, 0, -y_{n-2} .. -y_1): Z_k = -2i sum_i y_i sin(pi i k/(n-1)).
// Two real sequences a, b travel as a + ib: sum_a = -Im Z_k / 2, sum_b = Re Z_k / 2.
// The 2-D transform is T x T (rows, then columns); the spectrum is real and
// column-blocked like the DCT spectrum.  T is not orthogonal: the weights
// need no 1/n^2 and the 4-NS solve (spectral sums) does not apply.

// odd-extension position i of a length-M transform -> (source index j in
// 1..n-2, sign), j = 0 for the two zero positions
__device__ __forceinline__ int ar_src(int i, int n, int M, int* neg) {
  if (i >= 1 && i <= n - 2) { *neg = 0; return i; }
  if (i >= n) { *neg = 1; return M - i; }
  *neg = 0;
  return 0;
}

// rows: INV = false applies T^{-1} to the rows of buf[slot] (n x n) into the
// blocked spectrum S; INV = true applies T to the rows of S into buf[slot]
template <typename T, bool INV>
__global__ void __launch_bounds__(tr_nt(sizeof(T)), tr_minb(sizeof(T)))
k_ar_rows(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
          int slot, int pcg) {
  using T2 = typename Vec2<T>::type;
  constexpr int NT = tr_nt(sizeof(T));
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  if (tr_skip(states[item.x], pcg)) return;
  const int n = pd.n, M = pd.nfft, G = pd.row_g, TSg = fpad(M) + 1, cb = pd.cb;
  const int row0 = 2 * item.y * G;
  T* S = static_cast<T*>(pd.buf[SL_S]);
  T* X = static_cast<T*>(pd.buf[slot]);
  const T inv_n1 = T(1) / T(n - 1);
  const FastDiv fcb(cb);
  auto sidx = [&](int r, int k) -> size_t {
    const int b = fcb.div(k);
    return (size_t)b * n * cb + (size_t)r * cb + (k - b * cb);
  };
  // input row r at column k (0 past the last row)
  auto in = [&](int r, int k) -> T {
    if (r >= n) return T(0);
    return INV ? S[sidx(r, k)] : X[(size_t)r * n + k];
  };
  const FastDiv fM(M), fn(n);
  for (int e = threadIdx.x; e < G * M; e += NT) {
    const int g = fM.div(e), i = e - g * M;
    const int ra = row0 + 2 * g, rb = ra + 1;
    int neg;
    const int j = ar_src(i, n, M, &neg);
    T2 z;
    z.x = T(0); z.y = T(0);
    if (j) {
      if (INV) {
        z.x = in(ra, j); z.y = in(rb, j);
      } else {
        const T t = T(j) * inv_n1;
        z.x = in(ra, j) - in(ra, 0) * (T(1) - t) - in(ra, n - 1) * t;
        z.y = in(rb, j) - in(rb, 0) * (T(1) - t) - in(rb, n - 1) * t;
      }
      if (neg) { z.x = -z.x; z.y = -z.y; }
    }
    sm[g * TSg + fpad(i)] = z;
  }
  __syncthreads();
  fft_smem<T2, false>(G, pd);
  for (int e = threadIdx.x; e < G * n; e += NT) {
    const int g = fn.div(e), k = e - g * n;
    const int ra = row0 + 2 * g, rb = ra + 1;
    T va, vb;
    if (k == 0 || k == n - 1) {
      va = in(ra, k); vb = in(rb, k);
    } else {
      const T2 Z = sm[g * TSg + fpad(k)];
      if (INV) {
        const T t = T(k) * inv_n1;
        va = T(-0.5) * Z.y + in(ra, 0) * (T(1) - t) + in(ra, n - 1) * t;
        vb = T(0.5) * Z.x + in(rb, 0) * (T(1) - t) + in(rb, n - 1) * t;
      } else {
        va = -Z.y * inv_n1;
        vb = Z.x * inv_n1;
      }
    }
    if (INV) {
      if (ra < n) X[(size_t)ra * n + k] = va;
      if (rb < n) X[(size_t)rb * n + k] = vb;
    } else {
      if (ra < n) S[sidx(ra, k)] = va;
      if (rb < n) S[sidx(rb, k)] = vb;
    }
  }
}

// columns of one spectrum block: T^{-1}, the weight w = 1/(Lambda^2 + alpha)
// (Eq. Alg1, Alg3) or Lambda/(Lambda^2 + alpha) (Eq. Alg4), T; real columns
// 2g and 2g + 1 of the block travel as transform g
template <typename T, int mode>
__global__ void __launch_bounds__(tr_nt(sizeof(T)), tr_minb(sizeof(T)))
k_ar_cols(const Prob* __restrict__ probs, State* __restrict__ states, const int2* __restrict__ items,
          int pcg, double op_alpha, int op_kind) {
  using T2 = typename Vec2<T>::type;
  constexpr int NT = tr_nt(sizeof(T));
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int2 item = items[blockIdx.x];
  const Prob& pd = probs[item.x];
  if (tr_skip(states[item.x], pcg)) return;
  const int n = pd.n, M = pd.nfft, cb = pd.cb, TSg = fpad(M) + 1;
  const int G = cb / 2;
  T2* ends = sm + G * TSg;                     // weighted c_0 and c_{n-1} of each transform
  double alpha = pd.alpha;
  int kind = (pd.precond == P_TIKH) ? W_TIKH : W_INV;
  if (mode == COL_OP) { alpha = op_alpha; kind = op_kind; }
  const T Ta = T(alpha);
  const size_t base = (size_t)item.y * n * cb;
  const int kb = item.y * cb;
  T* S = static_cast<T*>(pd.buf[SL_S]) + base;
  const T inv_n1 = T(1) / T(n - 1);
  auto col_ok = [&](int c) { return kb + c < n; };
  auto in = [&](int r, int c) -> T { return col_ok(c) ? S[(size_t)r * cb + c] : T(0); };
  const FastDiv fM(M), fn(n);
  // 1. T^{-1} along the columns: odd extension of the detrended inner part
  for (int e = threadIdx.x; e < G * M; e += NT) {
    const int g = fM.div(e), i = e - g * M;
    const int ca = 2 * g, cbb = ca + 1;
    int neg;
    const int j = ar_src(i, n, M, &neg);
    T2 z;
    z.x = T(0); z.y = T(0);
    if (j) {
      const T t = T(j) * inv_n1;
      z.x = in(j, ca) - in(0, ca) * (T(1) - t) - in(n - 1, ca) * t;
      z.y = in(j, cbb) - in(0, cbb) * (T(1) - t) - in(n - 1, cbb) * t;
      if (neg) { z.x = -z.x; z.y = -z.y; }
    }
    sm[g * TSg + fpad(i)] = z;
  }
  __syncthreads();
  fft_smem<T2, false>(G, pd);
  // 2. coefficients, weighted; the odd extension of the weighted inner part
  //    replaces the spectrum in place (position k is read only by its own
  //    thread, and the mirror positions n .. M-1 are read by none)
  auto w = [&](int r, int c) -> T {
    return col_ok(c) ? weight_dct<T>(pd, base + (size_t)r * cb + c, Ta, T(1), kind) : T(0);
  };
  for (int e = threadIdx.x; e < G * n; e += NT) {
    const int g = fn.div(e), k = e - g * n;
    const int ca = 2 * g, cbb = ca + 1;
    T2* tb = sm + g * TSg;
    if (k == 0 || k == n - 1) {
      T2 v;
      v.x = in(k, ca) * w(k, ca);
      v.y = in(k, cbb) * w(k, cbb);
      ends[2 * g + (k == 0 ? 0 : 1)] = v;
      tb[fpad(k)] = mk2<T2>(T(0), T(0));
    } else {
      const T2 Z = tb[fpad(k)];
      T2 v;
      v.x = -Z.y * inv_n1 * w(k, ca);
      v.y = Z.x * inv_n1 * w(k, cbb);
      tb[fpad(k)] = v;
      tb[fpad(M - k)] = mk2<T2>(-v.x, -v.y);
    }
  }
  __syncthreads();
  // 3. T along the columns
  fft_smem<T2, false>(G, pd);
  for (int e = threadIdx.x; e < G * n; e += NT) {
    const int g = fn.div(e), k = e - g * n;
    const int ca = 2 * g, cbb = ca + 1;
    const T2 e0 = ends[2 * g], e1 = ends[2 * g + 1];
    T va, vb;
    if (k == 0) { va = e0.x; vb = e0.y; }
    else if (k == n - 1) { va = e1.x; vb = e1.y; }
    else {
      const T2 Z = sm[g * TSg + fpad(k)];
      const T t = T(k) * inv_n1;
      va = T(-0.5) * Z.y + e0.x * (T(1) - t) + e1.x * t;
      vb = T(0.5) * Z.x + e0.y * (T(1) - t) + e1.y * t;
    }
    if (col_ok(ca)) S[(size_t)k * cb + ca] = va;
    if (col_ok(cbb)) S[(size_t)k * cb + cbb] = vb;
  }
}

#ifndef MLBA_BODIES_ONLY  // launchers: not in the persistent kernel's unit
// ---------------------------------------------------------------------------
// Set-up: eigenvalues of C in FP64 (Section 4.1).  Q(dy, k2) = sum_dx h
// e^{-2 pi i k2 dx/n} (DFT) or sum_dx h cos(pi k2 dx/n) (DCT) comes from
// the host; here lambda(k1,k2) = sum_dy e^{-2 pi i k1 dy / n} Q(dy, k2) or
// sum_dy cos(pi k1 dy/n) Q(dy,k2), with tab the exact table of
// e^{-2 pi i m/n} (DFT, m < n) or cos(pi m/n) (DCT, m < 2n).  lambda and
// |lambda|^2 are rounded once to T and stored column-blocked; padding
// columns of the last block get lambda = 0, |lambda|^2 = 1.
__global__ void k_spectrum(int transform, int n, int p, int half, int cb,
                           const double* __restrict__ q, const double* __restrict__ tab,
                           void* lam, void* sigT, int is_double) {
  const int c = (p - 1) / 2;
  const int W = (transform == TR_DCT || transform == TR_AR) ? n : half;
  const int nb = (W + cb - 1) / cb;
  const size_t tot = (size_t)nb * n * cb;
  for (size_t L = blockIdx.x * (size_t)blockDim.x + threadIdx.x; L < tot;
       L += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(L / ((size_t)n * cb));
    const int rem = (int)(L - (size_t)b * n * cb);
    const int k1 = rem / cb, k2 = b * cb + (rem - k1 * cb);
    double re = 0.0, im = 0.0;
    if (k2 < W) {
      if (transform == TR_AR) {
        // angles k pi/(n-1), 0 for the two linear basis vectors (k = 0, n-1);
        // tab[m] = cos(pi m/(n-1)), m < 2(n-1)
        const int kk = (k1 == n - 1) ? 0 : k1, per = 2 * (n - 1);
        for (int a = 0; a < p; ++a) {
          int m = (kk * (a - c)) % per; if (m < 0) m += per;
          re += tab[m] * q[(size_t)a * n + k2];
        }
      } else if (transform == TR_DCT) {
        for (int a = 0; a < p; ++a) {
          int m = (k1 * (a - c)) % (2 * n); if (m < 0) m += 2 * n;
          re += tab[m] * q[(size_t)a * n + k2];
        }
      } else {
        for (int a = 0; a < p; ++a) {
          int m = (k1 * (a - c)) % n; if (m < 0) m += n;
          const double er = tab[2 * m], ei = tab[2 * m + 1];
          const double qr = q[2 * ((size_t)a * half + k2)], qi = q[2 * ((size_t)a * half + k2) + 1];
          re += er * qr - ei * qi;
          im += er * qi + ei * qr;
        }
      }
    }
    const double s2 = (k2 < W) ? re * re + im * im : 1.0;
    if (transform == TR_DCT || transform == TR_AR) {
      if (is_double) static_cast<double*>(lam)[L] = re;
      else static_cast<float*>(lam)[L] = (float)re;
    } else {
      if (is_double) static_cast<double2*>(lam)[L] = make_double2(re, im);
      else static_cast<float2*>(lam)[L] = make_float2((float)re, (float)im);
    }
    if (is_double) static_cast<double*>(sigT)[L] = s2;
    else static_cast<float*>(sigT)[L] = (float)s2;
  }
}

// ---------------------------------------------------------------------------
template <typename T>
void launch_rows_fwd(const Prob* probs, State* states, const int2* items, int nitems, int src,
                     int pcg, size_t smem, cudaStream_t s) {
  if (nitems > 0) k_rows_fwd<T><<<nitems, tr_nt(sizeof(T)), smem, s>>>(probs, states, items, src, pcg);
}
template <typename T>
void launch_cols(const Prob* probs, State* states, const int2* items, int nitems, int mode,
                 int pcg, double op_alpha, int op_kind, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return;
  const int nt = tr_nt(sizeof(T));
  if (mode == COL_FUSED)
    k_cols<T, COL_FUSED><<<nitems, nt, smem, s>>>(probs, states, items, pcg, op_alpha, op_kind);
  else if (mode == COL_FWD)
    k_cols<T, COL_FWD><<<nitems, nt, smem, s>>>(probs, states, items, pcg, op_alpha, op_kind);
  else if (mode == COL_NS_INV)
    k_cols<T, COL_NS_INV><<<nitems, nt, smem, s>>>(probs, states, items, pcg, op_alpha, op_kind);
  else
    k_cols<T, COL_OP><<<nitems, nt, smem, s>>>(probs, states, items, pcg, op_alpha, op_kind);
}
template <typename T>
void launch_rows_inv(const Prob* probs, State* states, const int2* items, int nitems, int dst,
                     int pcg, size_t smem, cudaStream_t s) {
  if (nitems > 0) k_rows_inv<T><<<nitems, tr_nt(sizeof(T)), smem, s>>>(probs, states, items, dst, pcg);
}
template <typename T>
void launch_ar_rows(const Prob* probs, State* states, const int2* items, int nitems, int slot,
                    int inv, int pcg, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return;
  if (inv) k_ar_rows<T, true><<<nitems, tr_nt(sizeof(T)), smem, s>>>(probs, states, items, slot, pcg);
  else k_ar_rows<T, false><<<nitems, tr_nt(sizeof(T)), smem, s>>>(probs, states, items, slot, pcg);
}
template <typename T>
void launch_ar_cols(const Prob* probs, State* states, const int2* items, int nitems, int mode,
                    int pcg, double op_alpha, int op_kind, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return;
  if (mode == COL_OP)
    k_ar_cols<T, COL_OP><<<nitems, tr_nt(sizeof(T)), smem, s>>>(probs, states, items, pcg, op_alpha, op_kind);
  else
    k_ar_cols<T, COL_FUSED><<<nitems, tr_nt(sizeof(T)), smem, s>>>(probs, states, items, pcg, op_alpha, op_kind);
}
template <typename T>
void launch_spec(const Prob* probs, State* states, const int2* items, int nitems, int cand,
                 cudaStream_t s) {
  if (nitems <= 0) return;
  if (cand) k_spec_cand<T><<<nitems, NS_NT, 0, s>>>(probs, states, items);
  else k_spec<T><<<nitems, NS_NT, 0, s>>>(probs, states, items);
}
void launch_spectrum_setup(int transform, int n, int p, int half, int cb, const double* q_dev,
                           const double* tab_dev, void* lam, void* sigT, int is_double,
                           cudaStream_t s) {
  const int W = (transform == TR_DCT || transform == TR_AR) ? n : half;
  const size_t tot = (size_t)((W + cb - 1) / cb) * n * cb;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_spectrum<<<blocks, 256, 0, s>>>(transform, n, p, half, cb, q_dev, tab_dev, lam, sigT, is_double);
}
template <typename T>
cudaError_t fft_set_smem(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_rows_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  for (const void* f : {(const void*)k_cols<T, COL_FUSED>, (const void*)k_cols<T, COL_FWD>,
                        (const void*)k_cols<T, COL_NS_INV>, (const void*)k_cols<T, COL_OP>}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  for (const void* f : {(const void*)k_ar_rows<T, false>, (const void*)k_ar_rows<T, true>,
                        (const void*)k_ar_cols<T, COL_FUSED>, (const void*)k_ar_cols<T, COL_OP>}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_rows_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define INST(T)                                                                                   \
  template void launch_rows_fwd<T>(const Prob*, State*, const int2*, int, int, int, size_t, cudaStream_t); \
  template void launch_cols<T>(const Prob*, State*, const int2*, int, int, int, double, int, size_t, cudaStream_t); \
  template void launch_rows_inv<T>(const Prob*, State*, const int2*, int, int, int, size_t, cudaStream_t); \
  template void launch_spec<T>(const Prob*, State*, const int2*, int, int, cudaStream_t);         \
  template void launch_ar_rows<T>(const Prob*, State*, const int2*, int, int, int, int, size_t, cudaStream_t); \
  template void launch_ar_cols<T>(const Prob*, State*, const int2*, int, int, int, double, int, size_t, cudaStream_t); \
  template cudaError_t fft_set_smem<T>(size_t);
INST(float)
INST(double)
#undef INST

#endif  // MLBA_BODIES_ONLY

}  // namespace mlba
