// Host launchers of the vector kernels (blas.cu).
#pragma once
#include "lqcd_internal.h"

namespace lqcd {
void v_norm2(int prec, const void* x, const VGeom& vg, const SegInfo* si, int nseg, double* partial, double* out,
             cudaStream_t st);
void v_convert(int pin, int pout, const void* in, void* out, const VGeom& vg, const SegInfo* si, int nseg,
               const double* scale, cudaStream_t st);
void v_axpy_mixed(int pe, void* x, const void* e, const VGeom& vg, const SegInfo* si, int nseg, const double* scale,
                  const int* active, cudaStream_t st);
void v_zero(int prec, void* x, const VGeom& vg, cudaStream_t st);
void v_copy(int prec, const void* a, void* b, const VGeom& vg, cudaStream_t st);
void bicg_init(int prec, const void* b, void* r, void* p, void* x, const VGeom& vg, const SegInfo* si, int nseg,
               double* partial, const KState& ks, const double* delta, const int* outer_active, cudaStream_t st);
void bicg_alpha(int prec, const void* r0, const void* v, const VGeom& vg, const SegInfo* si, int nseg,
                double* partial, const KState& ks, cudaStream_t st);
void bicg_s(int prec, const void* r, const void* v, void* s, const VGeom& vg, const SegInfo* si, int nseg,
            const KState& ks, cudaStream_t st);
void bicg_omega(int prec, const void* t, const void* s, const VGeom& vg, const SegInfo* si, int nseg,
                double* partial, const KState& ks, cudaStream_t st);
void bicg_fin_alpha_only(const double* partial, const VGeom& vg, const SegInfo* si, int nseg, const KState& ks,
                         cudaStream_t st);
void bicg_fin_omega_only(const double* partial, const VGeom& vg, const SegInfo* si, int nseg, const KState& ks,
                         cudaStream_t st);
void bicg_xr(int prec, void* x, const void* p, const void* s, const void* t, void* r, const void* r0,
             const VGeom& vg, const SegInfo* si, int nseg, double* partial, const KState& ks, cudaStream_t st);
void bicg_p(int prec, void* p, const void* r, const void* v, const VGeom& vg, const SegInfo* si, int nseg,
            const KState& ks, cudaStream_t st);
void count_active(const int* active, int n, int* count, cudaStream_t st);
void outer_update(const double* r2, const double* b2, int nsys, double tol, double inner_tol, int* active,
                  double* delta, double* scale, double* rel, int first, cudaStream_t st);
void recip(const double* a, double* b, int n, cudaStream_t st);
}  // namespace lqcd
