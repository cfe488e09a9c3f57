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

// One row MPO applied to an MPS.  Sparse projector form by default; with
// `dense` the columns are given as dense tensors Wd[c] = [bl][br][out][in]
// (used for the transposed MPO of the top-down pass and for the gradient
// sandwiches, on instances whose interfaces are small).
struct RowCtx {
  sgtn_inst* h = nullptr;
  int r = 0;
  const MPS* A = nullptr;       // the MPS being multiplied (left-canonical in row_step_ctx)
  std::vector<double*> Ahat;    // sparse: per column [nA][chl][chr]
  bool dense = false;
  bool transposed = false;      // dense and the MPO is T_r^T (out = sigma, in = u)
  std::vector<double*> Wd;      // dense: per column
  const Column& col(int c) const { return h->cols[r * h->M.C + c]; }
  int chl(int c) const { return A->bond[c]; }
  int chr(int c) const { return A->bond[c + 1]; }
  int nout(int c) const { return transposed ? col(c).nSig : col(c).nU; }
  int nin(int c) const { return transposed ? col(c).nU : col(c).nSig; }
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
// dense implementations (grad.cu)
double* theta_dense(RowCtx& X, int c, const double* K, int kp);
double* update_L_dense(RowCtx& X, int c, const double* L, const Ten& phi);

}  // namespace detail
}  // namespace sgtn
