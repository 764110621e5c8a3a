// Density-response moments in the auxiliary basis, FP64 path.
//
// TDA (Sec. II C, Eqs. 32-33):  T(0) = V,  T(n+1) = T(n) o D + 2 W(n) V
// RPA (Sec. II B, Eqs. 23-30):  T(0) = eta~(0) by quadrature,  T(1) = V o D,
//                               T(n) = T(n-2) o D^2 + 4 W(n-2) (V o D)
// with W(n) = T(n) V^T (the aux-basis factor of Eq. 15).  "o D" scales the
// columns ia by D_ia.  Each order is two GEMMs: W(n) (naux x naux, K = ov)
// and the update, whose epilogue applies the diagonal term in place, so T
// is read and written once per order and no intermediate is stored.
//
// With precision MGW_FP64_TC both GEMMs of an order run as FP64-accurate
// digit-sliced products on the tensor cores (ozaki.h): V is sliced once as
// rows (for W = T V^T) and, for TDA, once transposed (for W V); T and W(t)
// are sliced before each use, and the update's epilogue applies the
// diagonal term exactly as the FP64 kernel does.  With MGW_MIXED (TDA) V is
// first rounded to one 16-bit fixed-point grid (V', two digits per element)
// and the whole recursion runs on V' (T(0) = V' too), so the moments are
// exactly those of the system with V' at 13 digit products per product.
// For the RPA the contractions of the eta~(0) quadrature run on the tensor
// cores as well; the Cholesky solves of each node stay FP64 (cuSOLVER).
#include "mgw_internal.h"
#include "ozaki.h"
#include "ozaki_mixed.h"
#include "tc_gemm.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mgw {

// W = T V^T : A = T [naux][ov] row-major, B(k=ia, n=Q) = V[Q][ia]
static mgw_status w_gemm(mgw_handle* h, int naux, long ov, const double* T, const double* V, double* W) {
  // W(t) is symmetric: upper-triangle tiles only, mirrored in the epilogue
  return dgemm<64, 64>(h, naux, naux, ov, 1, ARowMajor{T, ov, 0}, BNMajor{V, ov, 0},
                       EpiStore{W, naux, 0, 1.0, 0.0}, "w_gemm", /*tri=*/1);
}

// T = T o d + alpha * W B : A = W [naux][naux], B = [naux][ov] row-major
static mgw_status t_update(mgw_handle* h, int naux, long ov, const double* W, const double* B,
                           double* T, const double* d, double alpha) {
  return dgemm<64, 64>(h, naux, ov, naux, 1, ARowMajor{W, naux, 0}, BRowMajor{B, ov, 0},
                       EpiDiagUpdate{T, ov, d, alpha}, "t_update");
}

// The contractions of the RPA path, on the FP64 units or, with `tc`, as
// FP64-accurate digit-sliced products on the tensor cores (ozaki.h): V is
// sliced once as rows (the B of every A V^T); A operands are sliced into
// `ad` and transposed B operands into `bd` right before each product.
struct RpaProducts {
  mgw_handle* h;
  int naux;
  long ov;
  const double* V;
  bool tc;
  int* dstatus;
  double *ad, *bd;
  oz::Sliced sv;
  CUtensorMap mv;

  // C [naux][naux] = alpha A V^T + beta C, A [naux][ov]
  mgw_status nt(double alpha, const double* A, double beta, double* C) const {
    if (!tc) return gemm_nt(h, naux, naux, ov, alpha, A, ov, V, ov, beta, C, naux);
    oz::Sliced sa;
    CUtensorMap ma;
    oz::place_sliced(ad, naux, ov, sa);
    MGW_TRY(oz::slice_rows(h, naux, ov, A, ov, sa));
    MGW_TRY(oz::digit_map(h, &ma, sa, oz::BM));
    return oz::ozaki_launch(h, ma, mv, sa.exps, sv.exps, naux, naux, (int)ov, oz::ARowsPlain{},
                            oz::EpiElem<oz::FStore>{oz::FStore{C, naux, alpha, beta}}, dstatus, "rpa_nt_tc");
  }
  // slices A [naux][naux] as rows and B [naux][ov] as columns (rows ia, K = Q)
  mgw_status slice_nn(const double* A, const double* B, oz::Sliced& sa, oz::Sliced& sb, CUtensorMap& ma,
                      CUtensorMap& mb) const {
    oz::place_sliced(ad, naux, naux, sa);
    MGW_TRY(oz::slice_rows(h, naux, naux, A, naux, sa));
    oz::place_sliced(bd, ov, naux, sb);
    MGW_TRY(oz::slice_cols(h, ov, naux, B, ov, sb));
    MGW_TRY(oz::digit_map(h, &ma, sa, oz::BM));
    return oz::digit_map(h, &mb, sb, oz::BN);
  }
  // C [naux][ov] = alpha A B + beta C, A [naux][naux], B [naux][ov]
  mgw_status nn(double alpha, const double* A, const double* B, double beta, double* C) const {
    if (!tc) return gemm_nn(h, naux, ov, naux, alpha, A, naux, B, ov, beta, C, ov);
    oz::Sliced sa, sb;
    CUtensorMap ma, mb;
    MGW_TRY(slice_nn(A, B, sa, sb, ma, mb));
    return oz::ozaki_launch(h, ma, mb, sa.exps, sb.exps, naux, (int)ov, naux, oz::ARowsPlain{},
                            oz::EpiElem<oz::FStore>{oz::FStore{C, ov, alpha, beta}}, dstatus, "rpa_nn_tc");
  }
  // T = T o d + alpha A B, A [naux][naux], B [naux][ov]
  mgw_status upd(const double* A, const double* B, double* T, const double* d, double alpha) const {
    if (!tc) return t_update(h, naux, ov, A, B, T, d, alpha);
    oz::Sliced sa, sb;
    CUtensorMap ma, mb;
    MGW_TRY(slice_nn(A, B, sa, sb, ma, mb));
    return oz::ozaki_launch(h, ma, mb, sa.exps, sb.exps, naux, (int)ov, naux, oz::ARowsPlain{},
                            oz::EpiElem<oz::FDiagUpdate>{oz::FDiagUpdate{T, ov, d, alpha}}, dstatus, "t_update_tc");
  }
};

// ---------------------------------------------------------------------------
// Quadrature for Eqs. 24-25: Clenshaw-Curtis on x in [-1, 1] with nq + 1
// points (x_k = cos(k pi / nq)), mapped to z = a (1 + x)/(1 - x) with
// a = sqrt(D_min D_max); the x = 1 node (z = infinity, where both
// integrands vanish) is dropped.  Weights are the closed cosine-sum form of
// the Clenshaw-Curtis weights times dz/dx = 2a/(1-x)^2.
static void quadrature(int nq, double dmin, double dmax, std::vector<double>& z, std::vector<double>& w) {
  const double pi = 3.14159265358979323846;
  const double a = std::sqrt(dmin * dmax);
  z.clear();
  w.clear();
  for (int k = 1; k <= nq; ++k) {
    double x = std::cos(k * pi / nq);
    double s = 0.0;
    for (int j = 1; j <= nq / 2; ++j) {
      double b = (j == nq / 2) ? 1.0 : 2.0;
      s += b / (4.0 * j * j - 1.0) * std::cos(2.0 * j * k * pi / nq);
    }
    double c = (k == nq) ? 1.0 : 2.0;
    double wx = c / nq * (1.0 - s);
    z.push_back(a * (1.0 + x) / (1.0 - x));
    w.push_back(wx * 2.0 * a / ((1.0 - x) * (1.0 - x)));
  }
}

// elementwise column factors for one node: f = F D, F, D E, E
__global__ void k_node_factors(long ov, const double* D, double z, double* fFD, double* fF, double* fDE,
                               double* fE) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= ov) return;
  double d = D[i];
  double F = 1.0 / (d * d + z * z);
  double E = exp(-z * d);
  fFD[i] = F * d;
  fF[i] = F;
  fDE[i] = d * E;
  fE[i] = E;
}

__global__ void k_sub_inplace(long n, double* x, const double* y) {  // x -= y
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) x[i] -= y[i];
}
__global__ void k_recip_sq(long n, const double* D, double* r, double* d2) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) { r[i] = 1.0 / D[i]; d2[i] = D[i] * D[i]; }
}

// Vt [ov][naux] = V [naux][ov]^T through a 32 x 32 shared-memory tile
__global__ void k_transpose(int naux, long ov, const double* __restrict__ V, double* __restrict__ Vt) {
  __shared__ double t[32][33];
  const long c0 = (long)blockIdx.x * 32, r0 = (long)blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long r = r0 + j, c = c0 + threadIdx.x;
    t[j][threadIdx.x] = (r < naux && c < ov) ? V[r * ov + c] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long c = c0 + j, r = r0 + threadIdx.x;
    if (c < ov && r < naux) Vt[c * naux + r] = t[threadIdx.x][j];
  }
}

// S [ov][bw] /= D[jb] + D[i0 + i]: the Cauchy factor of the exact G_offset
__global__ void k_cauchy_scale(long ov, int bw, long i0, const double* __restrict__ D, double* S) {
  const long n = ov * bw;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const long jb = idx / bw, i = idx % bw;
    S[idx] /= D[jb] + D[i0 + i];
  }
}
// G [naux][ov] columns i0.. += alpha X [naux][bw]
__global__ void k_add_block(int naux, long ov, int bw, long i0, double alpha, const double* __restrict__ X,
                            double* G) {
  const long n = (long)naux * bw;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const long p = idx / bw, i = idx % bw;
    G[p * ov + i0 + i] += alpha * X[idx];
  }
}

// G += 4 (V D)[(V^T V) o C], C_jb,ia = 1/(D_jb + D_ia): the z integral of
// Eq. 25 in closed form (int_0^inf e^{-z (D_jb + D_ia)} dz).  V^T V is
// formed and scaled one block of bw columns ia at a time (ov x bw), then
// multiplied by V D (in VD) into those columns of G: 4 ov^2 naux flops and
// ov bw doubles of scratch.  On the tensor cores both products are the
// FP64-accurate digit-sliced GEMM (V^T is formed once for the first).
static mgw_status g_offset_exact(mgw_handle* h, const RpaProducts& P, int naux, long ov, const double* V,
                                 const double* D, const double* VD, double* G) {
  const int bw = (int)std::min<long>(ov, 2048);
  double *S = nullptr, *X = nullptr, *Vt = nullptr;
  MGW_TRY(slot_buffer(h, 88, (size_t)ov * bw, &S));
  if (P.tc) {
    MGW_TRY(slot_buffer(h, 89, (size_t)naux * bw, &X));
    MGW_TRY(slot_buffer(h, 90, (size_t)ov * naux, &Vt));
    k_transpose<<<dim3((unsigned)((ov + 31) / 32), (unsigned)((naux + 31) / 32)), dim3(32, 8), 0, h->stream>>>(
        naux, ov, V, Vt);
    MGW_TRY(check_launch(h, "transpose"));
  }
  const unsigned gs = (unsigned)std::min<long>(((long)ov * bw + 255) / 256, 152L * 16);
  for (long i0 = 0; i0 < ov; i0 += bw) {
    const int nb = (int)std::min<long>(bw, ov - i0);
    if (P.tc) MGW_TRY(oz::gemm_fp64_tc_nn(h, (int)ov, nb, naux, Vt, naux, V + i0, ov, S, nb, "rpa_offset_vtv"));
    else MGW_TRY(gemm_tn(h, ov, nb, naux, 1.0, V, ov, V + i0, ov, 0.0, S, nb));
    k_cauchy_scale<<<gs, 256, 0, h->stream>>>(ov, nb, i0, D, S);
    MGW_TRY(check_launch(h, "cauchy_scale"));
    if (P.tc) {
      MGW_TRY(oz::gemm_fp64_tc_nn(h, naux, nb, (int)ov, VD, ov, S, nb, X, nb, "rpa_offset_g"));
      const unsigned ga = (unsigned)std::min<long>(((long)naux * nb + 255) / 256, 152L * 16);
      k_add_block<<<ga, 256, 0, h->stream>>>(naux, ov, nb, i0, 4.0, X, G);
      MGW_TRY(check_launch(h, "add_block"));
    } else {
      MGW_TRY(gemm_nn(h, naux, nb, ov, 4.0, VD, ov, S, nb, 1.0, G + i0, ov));
    }
  }
  return MGW_OK;
}

// eta~(0) of the RPA, Eqs. 23-28 (see the quadrature note above).
static mgw_status rpa_eta0(mgw_handle* h, const RpaProducts& P, int naux, long ov, int nq, bool exact_offset,
                           const double* V, const double* D, double dmin, double dmax, double* T0, double* work) {
  // work layout: G[naux*ov] B1[naux*ov] Q[naux^2] X[naux^2] IQ[naux^2] fac[4*ov]
  const long na2 = (long)naux * naux;
  double* G = work;
  double* B1 = G + naux * ov;
  double* Q = B1 + naux * ov;
  double* X = Q + na2;
  double* IQ = X + na2;
  double* fFD = IQ + na2;
  double* fF = fFD + ov;
  double* fDE = fF + ov;
  double* fE = fDE + ov;
  const double pi = 3.14159265358979323846;
  std::vector<double> z, w;
  quadrature(nq, dmin, dmax, z, w);
  const unsigned gov = (unsigned)((ov + 255) / 256);

  // G_offset starts at V D; in closed form it is completed here, else node by node below
  MGW_TRY(scale_columns(h, naux, ov, V, D, G));
  if (exact_offset) {
    MGW_TRY(scale_columns(h, naux, ov, V, D, B1));
    MGW_TRY(g_offset_exact(h, P, naux, ov, V, D, B1, G));
  }
  for (int j = 0; j < nq; ++j) {
    k_node_factors<<<gov, 256, 0, h->stream>>>(ov, D, z[j], fFD, fF, fDE, fE);
    MGW_TRY(check_launch(h, "node_factors"));
    // Q = 4 V F D V^T  (Eq. 26)
    MGW_TRY(scale_columns(h, naux, ov, V, fFD, B1));
    MGW_TRY(P.nt(4.0, B1, 0.0, Q));
    // X = Q (I + Q)^-1 - Q  (= Q((I+Q)^-1 - I), Eq. 24; Q and (I+Q)^-1 commute)
    MGW_CUDA(h, cudaMemcpyAsync(X, Q, sizeof(double) * na2, cudaMemcpyDeviceToDevice, h->stream));
    MGW_CUDA(h, cudaMemcpyAsync(IQ, Q, sizeof(double) * na2, cudaMemcpyDeviceToDevice, h->stream));
    MGW_TRY(add_identity(h, naux, IQ, 1.0));
    bool not_pd = false;
    MGW_TRY(potrf_potrs(h, naux, IQ, naux, X, &not_pd));
    k_sub_inplace<<<(unsigned)((na2 + 255) / 256), 256, 0, h->stream>>>(na2, X, Q);
    MGW_TRY(check_launch(h, "sub"));
    // G += (2/pi) w z^2 X (V F)   (integrand even in z: 1/pi over R = 2/pi over [0, inf))
    MGW_TRY(scale_columns(h, naux, ov, V, fF, B1));
    MGW_TRY(P.nn((2.0 / pi) * w[j] * z[j] * z[j], X, B1, 1.0, G));
    // G += 4 w (V D E V^T)(V E)   (Eq. 25)
    if (exact_offset) continue;
    MGW_TRY(scale_columns(h, naux, ov, V, fDE, B1));
    MGW_TRY(P.nt(1.0, B1, 0.0, Q));
    MGW_TRY(scale_columns(h, naux, ov, V, fE, B1));
    MGW_TRY(P.nn(4.0 * w[j], Q, B1, 1.0, G));
  }
  // eta~(0) = G D^-1 (I - 4 V^T (I + 4 V D^-1 V^T)^-1 V D^-1)   (Eq. 23)
  double* rD = fFD;
  double* d2 = fF;
  k_recip_sq<<<gov, 256, 0, h->stream>>>(ov, D, rD, d2);
  MGW_TRY(check_launch(h, "recip"));
  MGW_TRY(scale_columns(h, naux, ov, G, rD, T0));  // T0 = G D^-1
  MGW_TRY(scale_columns(h, naux, ov, V, rD, B1));  // B1 = V D^-1
  MGW_TRY(P.nt(4.0, B1, 0.0, Q));  // S - I
  MGW_TRY(add_identity(h, naux, Q, 1.0));
  MGW_TRY(P.nt(1.0, T0, 0.0, X));  // Y = G D^-1 V^T
  bool not_pd = false;
  MGW_TRY(potrf_potrs(h, naux, Q, naux, X, &not_pd));                      // X = Y S^-1
  MGW_TRY(P.nn(-4.0, X, B1, 1.0, T0));
  return MGW_OK;
}

__global__ void k_minmax(long n, const double* D, double* out) {
  // single block reduction of min and max
  __shared__ double smin[256], smax[256];
  double lo = 1e300, hi = -1e300;
  for (long i = threadIdx.x; i < n; i += blockDim.x) { lo = fmin(lo, D[i]); hi = fmax(hi, D[i]); }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = smin[0]; out[1] = smax[0]; }
}

}  // namespace mgw

using namespace mgw;

// The response from the FP64 particle-hole block Lov, or (Lq != null: TDA,
// MGW_MIXED) from the whole DF tensor on its grid as 16-bit integers with
// exponent eq, V' being its particle-hole block.
static mgw_status response_impl(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux, int nmom,
                                const double* eps_W, const double* Lov, const short* Lq, int eq, double* Wmom) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (nocc < 1 || nvir < 1 || naux < 1 || nmom < 1 || nmom > 64 || !eps_W || (!Lov && !Lq) || !Wmom)
    return fail(h, MGW_ERR_ARG, "mgw_response_moments: bad sizes or null pointer");
  if (Lq && (o->precision != MGW_MIXED || o->screening != MGW_TDA))
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_response_moments_q: the 16-bit grid tensor is the MGW_MIXED TDA input");
  if (o->screening != MGW_TDA && o->screening != MGW_RPA)
    return fail(h, MGW_ERR_ARG, "mgw_response_moments: unknown screening %d", o->screening);
  if (o->screening == MGW_RPA && (o->nquad < 2 || o->nquad % 2))
    return fail(h, MGW_ERR_ARG, "mgw_response_moments: nquad must be even and >= 2");
  if (o->precision != MGW_FP64 && o->precision != MGW_FP64_TC && o->precision != MGW_MIXED)
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_response_moments: precision %d not built", o->precision);
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long ov = (long)nocc * nvir;
  const long na2 = (long)naux * naux;
  const long tsz = (long)naux * ov;

  const bool any_tc = o->precision == MGW_FP64_TC || o->precision == MGW_MIXED;
  const bool use_tc = o->screening == MGW_TDA && any_tc;
  const bool rpa_tc = o->screening == MGW_RPA && any_tc;  // the RPA takes V unrounded in both modes
  // TDA under MGW_MIXED: the response of V' (V rounded to one 16-bit grid,
  // two digits): T(0) = V', W(t) = T(t) V'^T, T(t+1) = T(t) D + 2 W(t) V', so
  // W(t) = V' A'^t V'^T exactly for A' = D + 2 V'^T V'; T and W keep 7 digits
  const bool mixed = use_tc && o->precision == MGW_MIXED;
  const int vns = mixed ? oz::kGridSlices : oz::kSlices;
  Arena ar;
  double *D = nullptr, *T0 = nullptr, *T1 = nullptr, *aux = nullptr, *work = nullptr, *mm = nullptr;
  double *vd = nullptr, *vtd = nullptr, *td = nullptr, *wd = nullptr, *st = nullptr;
  ar.add(&D, ov);
  ar.add(&T0, tsz);
  ar.add(&mm, 2);
  // W(t) = T(t) V^T on the tensor cores: symmetric, so upper-triangle tiles
  // only, with K = ov split so that the kept tiles fill whole waves
  int w_req = 1, w_nz = 1;
  double* wpart = nullptr;
  const int wbn = mixed ? oz::kMBN : oz::BN;  // tile columns of the kernel that runs
  if (use_tc) {  // digit planes: V (rows Q, K = ov), V^T (rows ia, K = naux), T and W(t) per order
    int sms = 152;
    MGW_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    long kept = 0;
    for (int m0 = 0; m0 < naux; m0 += oz::BM)
      for (int n0 = 0; n0 < naux; n0 += wbn) kept += oz::sym_tile_lower(m0, n0, naux, wbn) ? 0 : 1;
    w_req = oz::best_split(kept, ov, sms);
    if (mixed) w_req = std::max(w_req, oz::mixed_min_split(ov));  // K per split within the mixed kernel's bound
    w_nz = oz::split_count(ov, w_req);
    ar.add(&vd, oz::sliced_doubles(naux, ov, vns));
    ar.add(&vtd, oz::sliced_doubles(ov, naux, vns));
    ar.add(&td, oz::sliced_doubles(naux, ov));
    ar.add(&wd, oz::sliced_doubles(naux, naux));
    ar.add(&st, 3);  // status word; the grid's max |V| and exponent
    if (w_nz > 1) ar.add(&wpart, (size_t)w_nz * na2);
  }
  double *ad = nullptr, *bd = nullptr;
  if (rpa_tc) {  // digit planes: V (rows Q, K = ov), A operands, transposed B operands
    ar.add(&vd, oz::sliced_doubles(naux, ov));
    ar.add(&ad, oz::sliced_doubles(naux, std::max<long>(ov, naux)));
    ar.add(&bd, oz::sliced_doubles(ov, naux));
    ar.add(&st, 1);
  }
  if (o->screening == MGW_RPA) {
    ar.add(&T1, tsz);
    ar.add(&aux, tsz + 2 * ov);  // V o D, D^2, spare
    ar.add(&work, 2 * tsz + 3 * na2 + 4 * ov);
  }
  MGW_TRY(ar.commit(h));
  MGW_TRY(energy_differences(h, nocc, nvir, eps_W, D));

  if (use_tc) {
    int* dstatus = h->defer_status ? h->defer_status : reinterpret_cast<int*>(st);
    if (!h->defer_status) MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
    oz::Sliced sv, svt, stt, sww;
    oz::place_sliced(vd, naux, ov, sv, vns);
    oz::place_sliced(vtd, ov, naux, svt, vns);
    oz::place_sliced(td, naux, ov, stt);
    oz::place_sliced(wd, naux, naux, sww);
    const oz::Gather gvt{ov + 1, 0, 1, naux + 1, 0, ov};  // V^T: rows ia, K = Q
    if (Lq) {
      // V' inside the whole tensor: element (Q, ia) at Lq[Q nmo^2 + i nmo + nocc + a]
      const long nmo = nocc + nvir, n2 = nmo * nmo;
      const short* Vq = Lq + nocc;
      MGW_TRY(oz::slice_gather_q(h, naux, ov, Vq, oz::Gather{naux + 1L, 0, n2, nvir, nmo, 1}, eq, sv));
      MGW_TRY(oz::slice_gather_q(h, ov, naux, Vq, oz::Gather{nvir, nmo, 1, naux + 1L, 0, n2}, eq, svt));
      MGW_TRY(oz::dequantize_gather(h, naux, ov, Vq, oz::Gather{naux + 1L, 0, n2, nvir, nmo, 1}, eq, T0));
    } else if (mixed) {
      int* gexp = reinterpret_cast<int*>(st + 2);
      MGW_TRY(oz::global_exponent(h, tsz, Lov, reinterpret_cast<unsigned long long*>(st + 1), gexp));
      MGW_TRY(oz::slice_rows_grid(h, naux, ov, Lov, ov, gexp, sv));
      MGW_TRY(oz::slice_gather_grid(h, ov, naux, Lov, gvt, gexp, svt));
      MGW_TRY(oz::round_to_grid(h, tsz, Lov, gexp, T0));  // T(0) = V'
    } else {
      MGW_TRY(oz::slice_rows(h, naux, ov, Lov, ov, sv));
      MGW_TRY(oz::slice_gather(h, ov, naux, Lov, gvt, svt));
      MGW_CUDA(h, cudaMemcpyAsync(T0, Lov, sizeof(double) * tsz, cudaMemcpyDeviceToDevice, h->stream));
    }
    CUtensorMap mv, mvt, mt, mw;
    MGW_TRY(oz::digit_map(h, &mv, sv, wbn));
    MGW_TRY(oz::digit_map(h, &mvt, svt, wbn));
    MGW_TRY(oz::digit_map(h, &mt, stt, oz::BM));
    MGW_TRY(oz::digit_map(h, &mw, sww, oz::BM));
    // the two products of an order: B = V (rows Q) or V^T (rows ia), 2 digits under MGW_MIXED
    auto launch = [&](const CUtensorMap& ma, const CUtensorMap& mb, const int* ea, const int* eb, int M, int N,
                      int K, auto epi, const char* what, int nsp) {
      if (mixed)
        return oz::ozaki_mixed_launch<true>(h, ma, mb, ea, eb, M, N, K, oz::ARowsPlain{}, epi, dstatus, what, nsp);
      return oz::ozaki_launch(h, ma, mb, ea, eb, M, N, K, oz::ARowsPlain{}, epi, dstatus, what, nsp);
    };
    for (int n = 0; n < nmom; ++n) {
      double* Wn = Wmom + (long)n * na2;
      MGW_TRY(oz::slice_rows(h, naux, ov, T0, ov, stt));
      if (w_nz == 1) {
        MGW_TRY(launch(mt, mv, stt.exps, sv.exps, naux, naux, (int)ov,
                       oz::EpiElem<oz::FStoreSym>{oz::FStoreSym{Wn, naux, 0}}, "w_gemm_tc", 1));
      } else {
        MGW_TRY(launch(mt, mv, stt.exps, sv.exps, naux, naux, (int)ov,
                       oz::EpiElem<oz::FStoreSym>{oz::FStoreSym{wpart, naux, na2}}, "w_gemm_tc", w_req));
        MGW_TRY(oz::reduce_splits(h, na2, w_nz, wpart, Wn, 0));
      }
      if (n + 1 < nmom) {
        MGW_TRY(oz::slice_rows(h, naux, naux, Wn, naux, sww));
        MGW_TRY(launch(mw, mvt, sww.exps, svt.exps, naux, (int)ov, naux,
                       oz::EpiElem<oz::FDiagUpdate>{oz::FDiagUpdate{T0, ov, D, 2.0}}, "t_update_tc", 1));
      }
    }
    return h->defer_status ? MGW_OK : tc::check_tc_status(h, dstatus, "mgw_response_moments");
  }

  if (o->screening == MGW_TDA) {
    MGW_CUDA(h, cudaMemcpyAsync(T0, Lov, sizeof(double) * tsz, cudaMemcpyDeviceToDevice, h->stream));
    for (int n = 0; n < nmom; ++n) {
      double* Wn = Wmom + (long)n * na2;
      MGW_TRY(w_gemm(h, naux, ov, T0, Lov, Wn));
      if (n + 1 < nmom) MGW_TRY(t_update(h, naux, ov, Wn, Lov, T0, D, 2.0));
    }
    return MGW_OK;
  }

  // RPA
  k_minmax<<<1, 256, 0, h->stream>>>(ov, D, mm);
  MGW_TRY(check_launch(h, "minmax"));
  double hmm[2];
  MGW_CUDA(h, cudaMemcpyAsync(hmm, mm, sizeof hmm, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (!(hmm[0] > 0.0))
    return fail(h, MGW_ERR_ARG, "mgw_response_moments: RPA needs D_ia > 0 (min D = %g)", hmm[0]);
  double* LD = aux;
  double* D2 = aux + tsz;
  double* rD = D2 + ov;
  k_recip_sq<<<(unsigned)((ov + 255) / 256), 256, 0, h->stream>>>(ov, D, rD, D2);
  MGW_TRY(check_launch(h, "recip"));
  MGW_TRY(scale_columns(h, naux, ov, Lov, D, LD));
  RpaProducts P{h, naux, ov, Lov, rpa_tc, nullptr, ad, bd, {}, {}};
  if (rpa_tc) {
    P.dstatus = h->defer_status ? h->defer_status : reinterpret_cast<int*>(st);
    if (!h->defer_status) MGW_CUDA(h, cudaMemsetAsync(P.dstatus, 0, sizeof(int), h->stream));
    oz::place_sliced(vd, naux, ov, P.sv);
    MGW_TRY(oz::slice_rows(h, naux, ov, Lov, ov, P.sv));
    MGW_TRY(oz::digit_map(h, &P.mv, P.sv, oz::BN));
  }
  MGW_TRY(rpa_eta0(h, P, naux, ov, o->nquad, o->rpa_offset != 0, Lov, D, hmm[0], hmm[1], T0, work));
  MGW_CUDA(h, cudaMemcpyAsync(T1, LD, sizeof(double) * tsz, cudaMemcpyDeviceToDevice, h->stream));
  double* T[2] = {T0, T1};
  for (int n = 0; n < nmom; ++n) {
    double* Wn = Wmom + (long)n * na2;
    if (n >= 2) MGW_TRY(P.upd(Wmom + (long)(n - 2) * na2, LD, T[n & 1], D2, 4.0));
    if (rpa_tc) MGW_TRY(P.nt(1.0, T[n & 1], 0.0, Wn));
    else MGW_TRY(w_gemm(h, naux, ov, T[n & 1], Lov, Wn));
  }
  if (rpa_tc && !h->defer_status) return tc::check_tc_status(h, P.dstatus, "mgw_response_moments");
  return MGW_OK;
}

extern "C" mgw_status mgw_response_moments(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux,
                                           int nmom, const double* eps_W, const double* Lov, double* Wmom) {
  if (!Lov) return h ? fail(h, MGW_ERR_ARG, "mgw_response_moments: null Lov") : MGW_ERR_ARG;
  return response_impl(h, o, nocc, nvir, naux, nmom, eps_W, Lov, nullptr, 0, Wmom);
}

extern "C" mgw_status mgw_response_moments_q(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux,
                                             int nmom, const double* eps_W, const short* Lq, int e, double* Wmom) {
  if (!Lq) return h ? fail(h, MGW_ERR_ARG, "mgw_response_moments_q: null Lq") : MGW_ERR_ARG;
  mgw_options m;
  if (o) m = *o;
  else mgw_options_default(&m);
  m.precision = MGW_MIXED;
  m.screening = MGW_TDA;
  return response_impl(h, &m, nocc, nvir, naux, nmom, eps_W, nullptr, Lq, e, Wmom);
}
