// Internal interface of the boundary-MPS row step (shared by the bottom-up
// contraction and the top-down pass used for gradients).
#pragma once
#include <vector>

#include "handle.h"

namespace sgtn {
namespace detail {

constexpr double RANK_TOL = 1e-12;

struct Ten {
  double* p = nullptr;
  int a = 1, u = 1, b = 1;   // [a][u][b]
  long long n() const { return (long long)a * u * b; }
};

struct SvdOut {
  int k = 0;
  double* US = nullptr;   // m x k
  double* Vt = nullptr;   // k x n
  double* dsig = nullptr; // k sigmas then k inverse sigmas (device)
  std::vector<double> sig;
  void release();
};

// One row MPO applied to an MPS, in the sparse projector form of its
// columns.  cols / w, when set, replace the row's columns and per-state
// weights (the top-down pass of the gradient applies the transposed MPO,
// written as forward-form columns over virtual states).
struct RowCtx {
  sgtn_inst* h = nullptr;
  int r = 0;
  const MPS* A = nullptr;       // the MPS being multiplied (left-canonical in row_step_ctx)
  std::vector<double*> Ahat;    // per column [nA][chl][chr]
  const Column* cols = nullptr;
  const double* const* w = nullptr;
  // per column: power-of-two exponent s of the weights in the FP32 / TF32 /
  // BF16 contractions (the site-diagram results are then 2^s times the true
  // ones; the log-scale bookkeeping takes s off).  Learned by the zipper,
  // kept across calls; unused in FP64.  nullptr: no scaling.
  int* sexp = nullptr;
  int* lexp = nullptr;   // the same for the left-environment updates (their scale is not kept)
  const Column& col(int c) const { return cols ? cols[c] : h->cols[r * h->M.C + c]; }
  const double* wts(int c) const { return w ? w[c] : h->ds[r * h->M.C + c].w; }
  int chl(int c) const { return A->bond[c]; }
  int chr(int c) const { return A->bond[c + 1]; }
  int nout(int c) const { return col(c).nU; }
  int nin(int c) const { return col(c).nSig; }
};

double* dmalloc(long long n);
void dfree(double*& p);
SvdOut svd(sgtn_inst* h, const double* Th, int m, int n, int cap);
void normalise(sgtn_inst* h, double* x, long long n, double& lognorm);
double norm_host(sgtn_inst* h, const double* x, long long n, bool allow_zero);
void left_canonical(sgtn_inst* h, MPS& A);
double* theta_of(RowCtx& X, int c, const double* K, int kp);
double* update_L(RowCtx& X, int c, const double* L, const Ten& phi);
double* update_R(RowCtx& X, int c, const double* ThR, const Ten& phi);
void row_step_ctx(RowCtx& X, MPS& A, int chi, int n_sweeps, MPS& out, double& worst);
void compute_ahat(RowCtx& X);
double norm_value(sgtn_inst* h, const double* x, long long n);
int exp_step(double v);
double* update_L_adapt(RowCtx& X, int c, const double* L, const Ten& phi);

}  // namespace detail
}  // namespace sgtn
