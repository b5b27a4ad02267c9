// Exact stabilizer-tableau -> statevector export (the STAB -> SV row of
// Table II): a tableau boundary of n <= 30 qubits becomes the dense state a
// statevector suffix continues from.
//
// 1) One thread turns the stored inverse tableau T(P) = C^-1 P C into the
//    stabilizer generators S_i = C Z_i C^-1 of the state C|0...0>.  For a
//    symplectic map the inverse is Omega M^T Omega, so S_i has X-part bit j
//    = x-bit i of T(Z_j) and Z-part bit j = x-bit i of T(X_j); its sign
//    follows from requiring T(S_i) = Z_i, evaluated as a product of rows.
//    The generators are brought to reduced echelon form on their X-parts
//    (k pivots); the n-k generators left with no X-part are +-Z strings
//    whose signs fix parities of the support; solving them gives a basis
//    state x0 in the support.
// 2) Every amplitude is then independent: x is in the support iff
//    w = x ^ x0 lies in the span of the k echelon X-parts (read off at the
//    pivot bits), and then psi[x] = 2^(-k/2) <x|G|x0> with G the product of
//    the selected generators, which is i^e (-1)^(z.x0).  The global phase
//    is fixed by psi[x0] = 2^(-k/2) > 0.
//
// Paulis are kept as i^e X^x Z^z (e mod 4):
//   (e1,x1,z1)(e2,x2,z2) = (e1 + e2 + 2 popc(z1 & x2), x1 ^ x2, z1 ^ z2);
// a tableau row (-1)^r i^{x.z} X^x Z^z has e = 2r + popc(x & z).
#include <cuda_runtime.h>

#include <algorithm>

#include "qw_internal.h"

namespace qw {

struct Pl {
  uint32_t e;
  uint64_t x, z;
};
template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };
__device__ __forceinline__ Pl pl_mul_d(const Pl &a, const Pl &b) {
  Pl r;
  r.e = (a.e + b.e + 2u * (uint32_t)__popcll(a.z & b.x)) & 3u;
  r.x = a.x ^ b.x;
  r.z = a.z ^ b.z;
  return r;
}

// rows: 2n rows of (x word, z word) (W = 1), sign bytes after them
__global__ void stab_basis_kernel(const uint64_t *__restrict__ rows, const uint8_t *__restrict__ sign,
                                  uint32_t n, StabBasis *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Pl T[2 * QW_SV_MAX_QUBITS];  // T(X_j) = T[j], T(Z_j) = T[n + j]
  for (uint32_t r = 0; r < 2 * n; r++) {
    const uint64_t x = rows[2 * r], z = rows[2 * r + 1];
    T[r].x = x;
    T[r].z = z;
    T[r].e = (2u * (sign[r] & 1u) + (uint32_t)__popcll(x & z)) & 3u;
  }
  Pl S[QW_SV_MAX_QUBITS];
  uint32_t err = 0;
  for (uint32_t i = 0; i < n; i++) {
    uint64_t u = 0, v = 0;
    for (uint32_t j = 0; j < n; j++) {
      u |= ((T[n + j].x >> i) & 1ull) << j;
      v |= ((T[j].x >> i) & 1ull) << j;
    }
    // T(H(u, v)) with H(u, v) = i^{u.v} X^u Z^v, as a product of rows
    Pl acc{(uint32_t)__popcll(u & v) & 3u, 0ull, 0ull};
    for (uint32_t j = 0; j < n; j++)
      if ((u >> j) & 1ull) acc = pl_mul_d(acc, T[j]);
    for (uint32_t j = 0; j < n; j++)
      if ((v >> j) & 1ull) acc = pl_mul_d(acc, T[n + j]);
    // acc must be i^e Z_i with e in {0, 2}; S_i = i^{-e} H(u, v)
    if (acc.x != 0ull || acc.z != (1ull << i) || (acc.e & 1u)) err = 1;
    S[i].x = u;
    S[i].z = v;
    S[i].e = ((uint32_t)__popcll(u & v) + (4u - acc.e)) & 3u;
  }
  // reduced echelon form on the X-parts
  uint32_t k = 0;
  uint8_t piv[QW_SV_MAX_QUBITS];
  for (uint32_t p = 0; p < n && k < n; p++) {
    uint32_t r = k;
    while (r < n && !((S[r].x >> p) & 1ull)) r++;
    if (r == n) continue;
    const Pl t = S[r];
    S[r] = S[k];
    S[k] = t;
    for (uint32_t q = 0; q < n; q++)
      if (q != k && ((S[q].x >> p) & 1ull)) S[q] = pl_mul_d(S[k], S[q]);
    piv[k] = (uint8_t)p;
    k++;
  }
  // the remaining generators are (-1)^{e/2} Z^z: parity z.x0 = e/2
  uint64_t zc[QW_SV_MAX_QUBITS];
  uint32_t cc[QW_SV_MAX_QUBITS];
  uint32_t m = 0;
  for (uint32_t q = k; q < n; q++) {
    if (S[q].x != 0ull || (S[q].e & 1u)) err = 1;
    zc[m] = S[q].z;
    cc[m] = (S[q].e >> 1) & 1u;
    m++;
  }
  // solve the parity system by elimination; free bits are 0
  uint32_t rank = 0;
  uint8_t zp[QW_SV_MAX_QUBITS];
  for (uint32_t p = 0; p < n && rank < m; p++) {
    uint32_t r = rank;
    while (r < m && !((zc[r] >> p) & 1ull)) r++;
    if (r == m) continue;
    uint64_t tz = zc[r];
    zc[r] = zc[rank];
    zc[rank] = tz;
    uint32_t tc = cc[r];
    cc[r] = cc[rank];
    cc[rank] = tc;
    for (uint32_t q = 0; q < m; q++)
      if (q != rank && ((zc[q] >> p) & 1ull)) { zc[q] ^= zc[rank]; cc[q] ^= cc[rank]; }
    zp[rank] = (uint8_t)p;
    rank++;
  }
  for (uint32_t q = rank; q < m; q++)
    if (cc[q]) err = 1;  // inconsistent parities: not a valid state
  uint64_t x0 = 0;
  for (uint32_t q = 0; q < rank; q++)
    if (cc[q]) x0 |= 1ull << zp[q];  // every other bit of row q is a free (zero) bit
  out->n = n;
  out->k = k;
  out->x0 = x0;
  out->err = err;
  for (uint32_t j = 0; j < k; j++) {
    out->gx[j] = S[j].x;
    out->gz[j] = S[j].z;
    out->ge[j] = S[j].e;
    out->piv[j] = piv[j];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) stab_export_kernel(const StabBasis *__restrict__ B, uint32_t n_eff,
                                                           typename Cx<T>::t *psi) {
  __shared__ StabBasis sb;
  if (threadIdx.x == 0) sb = *B;
  __syncthreads();
  const uint64_t dim = 1ull << n_eff;
  const double mag = exp2(-0.5 * (double)sb.k);
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < dim;
       x += (uint64_t)gridDim.x * blockDim.x) {
    typename Cx<T>::t a;
    a.x = 0;
    a.y = 0;
    if ((x >> sb.n) == 0ull && !sb.err) {
      uint64_t w = x ^ sb.x0;
      Pl acc{0u, 0ull, 0ull};
      for (uint32_t j = 0; j < sb.k; j++)
        if ((w >> sb.piv[j]) & 1ull) acc = pl_mul_d(acc, Pl{sb.ge[j], sb.gx[j], sb.gz[j]});
      if (acc.x == w) {
        const uint32_t e = (acc.e + 2u * (uint32_t)(__popcll(acc.z & sb.x0) & 1)) & 3u;
        // i^e: 1, i, -1, -i
        a.x = (T)((e == 0) ? mag : ((e == 2) ? -mag : 0.0));
        a.y = (T)((e == 1) ? mag : ((e == 3) ? -mag : 0.0));
      }
    }
    psi[x] = a;
  }
}

void launch_stab_export(const void *tableau, uint32_t n, StabBasis *basis, bool fp64, uint32_t n_eff, void *dst,
                        int sm_count, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t words = (size_t)2 * n * 2;  // 2n rows x (x, z), W = 1
  const uint64_t *rows = (const uint64_t *)tableau;
  const uint8_t *sign = (const uint8_t *)(rows + words);
  stab_basis_kernel<<<1, 32, 0, s>>>(rows, sign, n, basis);
  const uint64_t dim = 1ull << n_eff;
  const uint64_t want = (dim + 255) / 256;
  const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)sm_count * 16);
  if (fp64)
    stab_export_kernel<double><<<blocks, 256, 0, s>>>(basis, n_eff, (double2 *)dst);
  else
    stab_export_kernel<float><<<blocks, 256, 0, s>>>(basis, n_eff, (float2 *)dst);
}

}  // namespace qw
