// Device-resident AC-OPF model data (see opf.cu).
#pragma once
#include "common.cuh"

namespace cipm {

struct OpfData {
  int nb = 0, nbr = 0, ng = 0, n = 0, me = 0, mi = 0, ref = 0;
  int form = 0;  // 0: compact polar; 1: with branch-flow variables (see opf_dev.cuh)
  int *f_bus = nullptr, *t_bus = nullptr, *gen_bus = nullptr;
  double4_32a *adm = nullptr;  // per branch: G1, B1, G2, B2 (identical for both ends, unit tap)
  double *rate = nullptr, *pd = nullptr, *qd = nullptr, *c2 = nullptr, *c1 = nullptr;
  double *xl = nullptr, *xu = nullptr;  // variable bounds (+-inf where absent)
  int *J_rowptr = nullptr, *J_colind = nullptr, *W_rowptr = nullptr, *W_colind = nullptr;
  int nnzJ = 0, nnzW = 0;
  int *jentry = nullptr, *wentry = nullptr;  // model term -> value slot
  double *fpart = nullptr;
};

int opf_create(OpfData &M, int nb, int nbr, int ng, const int *f_bus, const int *t_bus,
               const double *r, const double *x, const double *b, const double *rate,
               const double *pd, const double *qd, const int *gen_bus, const double *c2,
               const double *c1, const double *xl, const double *xu, cudaStream_t s,
               int form = 0);
// x0 of the flow-variable form: each flow variable at the flow of the voltages in x (x[0, nc)
// already set)
int opf_flow_start(const OpfData &M, double *x, cudaStream_t s);
void opf_free(OpfData &M);
int opf_eval(const OpfData &M, const double *x, const double *y, const double *z, double sigma_f,
             double *f, double *grad, double *g, double *h, double *Jv, double *Wv,
             cudaStream_t s);

}  // namespace cipm

struct ipm_opf_s {
  cipm::OpfData M;
};
