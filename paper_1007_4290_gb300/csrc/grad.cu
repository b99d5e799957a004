#include "handle.h"
int hsw_grad(hsweep_s* h, const c128* f, int nsrc, const int* rec, int nrec, const c128* d,
             double* grad, double* misfit, double tol) { return HSWEEP_ERR_ARG; }
