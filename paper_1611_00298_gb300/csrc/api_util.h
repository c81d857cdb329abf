// Helpers shared by the C-ABI translation units.
#pragma once
#include "ops.h"

int fail(eofa_ctx* ctx, int code, const std::string& msg);
void check_ls(const eofa_ctx* ctx, int Ls);
void require_gauge(const eofa_ctx* ctx);

void apply_dwf_fields(eofa_ctx* ctx, const Coeffs& c, int dagger, const void* in_e, const void* in_o, void* out_e,
                      void* out_o, cudaStream_t st);
void apply_eofa_fields(eofa_ctx* ctx, const Op5& G, const void* in_e, const void* in_o, void* out_e, void* out_o,
                       cudaStream_t st);

// one solve on device canonical buffers (solver.cu)
int solve_dev_impl(eofa_ctx* ctx, const eofa_solve_params* p, const double* b_dev, double* x_dev,
                   eofa_solve_info* info, cudaStream_t st);

// Omega_chi P_chi phi: 4D canonical phi -> 5D canonical out (Omega on the device, Ls values)
void eofa_embed(eofa_ctx* ctx, const double* phi, const double* Om_dev, int chi, double* out, cudaStream_t st);

// gauge action (host value, synchronous) and force (= or += into F) on canonical links (gauge.cu)
double gauge_action_now(eofa_ctx* ctx, const double* U, double beta, cudaStream_t st);
void gauge_force_launch(eofa_ctx* ctx, const double* U, double beta, int accumulate, double* F, cudaStream_t st);

extern "C" int eofa_force_parts_dev(eofa_ctx* ctx, int Ls, double alpha, double M5, double m1, double m2,
                                    int precision, double tol, const double* phi_dev, double* FL_dev, double* FR_dev,
                                    eofa_solve_info info[2], void* stream);
