// mls_dispatch.cuh -- runtime dispatch of the templated MLS kernels. The definitions live
// in mls_inst_d2.cu / mls_inst_d3.cu so the two dimensions compile in parallel.
#pragma once

#include "mls_kernels.cuh"
#include "trace.cuh"

namespace pcms {

// assemble: mode MODE_COUNT / MODE_MAP / MODE_FUSED; G = lanes per target (8 or 32);
// field_double: FUSED field type (float or double)
#define PCMS_DECLARE_MLS_DISPATCH(DIMV)                                                       \
    void assemble_dispatch_d##DIMV(int deg, bool mixed, int mode, int G, bool field_double,   \
                                   const AsmArgs& a, int blocks, cudaStream_t s);             \
    void solve_dispatch_d##DIMV(int deg, int mode, bool mom_double, const SolveArgs& a,       \
                                int blocks, cudaStream_t s);                                  \
    void shape_dispatch_d##DIMV(int deg, bool mixed, int G, const ShapeArgs& a, int blocks,   \
                                cudaStream_t s);                                              \
    void assemble_comp_dispatch_d##DIMV(int deg, int mode, int G, const AsmArgs& a,            \
                                        int blocks, cudaStream_t s);
PCMS_DECLARE_MLS_DISPATCH(2)
PCMS_DECLARE_MLS_DISPATCH(3)

// compensated FP32 assembly (mixed precision, tier 2), MODE_MAP or MODE_FUSED
inline void assemble_comp_any(int dim, int deg, int mode, int G, const AsmArgs& a, int blocks,
                              cudaStream_t s) {
    PCMS_TRACE(mode == MODE_FUSED ? "mls_assemble_fused_comp" : "mls_assemble_map_comp", s);
    if (dim == 2) assemble_comp_dispatch_d2(deg, mode, G, a, blocks, s);
    else assemble_comp_dispatch_d3(deg, mode, G, a, blocks, s);
}

inline void assemble_any(int dim, int deg, bool mixed, int mode, int G, bool fd,
                         const AsmArgs& a, int blocks, cudaStream_t s) {
    static const char* names[2][3] = {
        {"mls_count_fp64", "mls_assemble_map_fp64", "mls_assemble_fused_fp64"},
        {"mls_count_mixed", "mls_assemble_map_mixed", "mls_assemble_fused_mixed"}};
    PCMS_TRACE(names[mixed ? 1 : 0][mode], s);
    if (dim == 2) assemble_dispatch_d2(deg, mixed, mode, G, fd, a, blocks, s);
    else assemble_dispatch_d3(deg, mixed, mode, G, fd, a, blocks, s);
}
inline void solve_any(int dim, int deg, int mode, bool md, const SolveArgs& a, int blocks,
                      cudaStream_t s) {
    PCMS_TRACE(mode == MODE_FUSED ? "mls_solve_fused" : "mls_solve_map", s);
    if (dim == 2) solve_dispatch_d2(deg, mode, md, a, blocks, s);
    else solve_dispatch_d3(deg, mode, md, a, blocks, s);
}
inline void shape_any(int dim, int deg, bool mixed, int G, const ShapeArgs& a, int blocks,
                      cudaStream_t s) {
    PCMS_TRACE(mixed ? "mls_shape_mixed" : "mls_shape_fp64", s);
    if (dim == 2) shape_dispatch_d2(deg, mixed, G, a, blocks, s);
    else shape_dispatch_d3(deg, mixed, G, a, blocks, s);
}

}  // namespace pcms

// Definitions for one dimension; included by exactly one .cu per dimension.
#define PCMS_DEFINE_MLS_DISPATCH(DIMV)                                                        \
    namespace pcms {                                                                          \
    template <int DEG, bool MIXED>                                                            \
    static void asm_mode(int mode, int G, bool fd, const AsmArgs& a, int b, cudaStream_t s) { \
        if (mode == MODE_COUNT) {                                                             \
            if (DEG != 0) return;                                                             \
            if (G == 32) k_assemble<DIMV, 0, MIXED, MODE_COUNT, 32, float><<<b, 256, 0, s>>>(a); \
            else k_assemble<DIMV, 0, MIXED, MODE_COUNT, 8, float><<<b, 256, 0, s>>>(a);       \
        } else if (mode == MODE_MAP) {                                                        \
            if (G == 32) k_assemble<DIMV, DEG, MIXED, MODE_MAP, 32, float><<<b, 256, 0, s>>>(a); \
            else k_assemble<DIMV, DEG, MIXED, MODE_MAP, 8, float><<<b, 256, 0, s>>>(a);       \
        } else {                                                                              \
            if (fd) {                                                                         \
                if (MIXED) return;                                                            \
                if (G == 32) k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 32, double><<<b, 256, 0, s>>>(a); \
                else k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 8, double><<<b, 256, 0, s>>>(a); \
            } else {                                                                          \
                if (G == 32) k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 32, float><<<b, 256, 0, s>>>(a); \
                else k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 8, float><<<b, 256, 0, s>>>(a);  \
            }                                                                                 \
        }                                                                                     \
    }                                                                                         \
    void assemble_dispatch_d##DIMV(int deg, bool mixed, int mode, int G, bool fd,               \
                                 const AsmArgs& a, int b, cudaStream_t s) {                   \
        if (mode == MODE_COUNT) deg = 0;                                                      \
        if (mixed) {                                                                          \
            if (deg == 0) asm_mode<0, true>(mode, G, fd, a, b, s);                            \
            else if (deg == 1) asm_mode<1, true>(mode, G, fd, a, b, s);                       \
            else asm_mode<2, true>(mode, G, fd, a, b, s);                                     \
        } else {                                                                              \
            if (deg == 0) asm_mode<0, false>(mode, G, fd, a, b, s);                           \
            else if (deg == 1) asm_mode<1, false>(mode, G, fd, a, b, s);                      \
            else asm_mode<2, false>(mode, G, fd, a, b, s);                                    \
        }                                                                                     \
        PCMS_LAUNCH_CHECK("k_assemble");                                                      \
    }                                                                                         \
    void solve_dispatch_d##DIMV(int deg, int mode, bool md, const SolveArgs& a, int b,          \
                              cudaStream_t s) {                                               \
        if (mode == MODE_FUSED) {                                                             \
            if (md) {                                                                         \
                if (deg == 0) k_solve<DIMV, 0, MODE_FUSED, double><<<b, 128, 0, s>>>(a);     \
                else if (deg == 1) k_solve<DIMV, 1, MODE_FUSED, double><<<b, 128, 0, s>>>(a); \
                else k_solve<DIMV, 2, MODE_FUSED, double><<<b, 128, 0, s>>>(a);              \
            } else {                                                                          \
                if (deg == 0) k_solve<DIMV, 0, MODE_FUSED, float><<<b, 128, 0, s>>>(a);      \
                else if (deg == 1) k_solve<DIMV, 1, MODE_FUSED, float><<<b, 128, 0, s>>>(a); \
                else k_solve<DIMV, 2, MODE_FUSED, float><<<b, 128, 0, s>>>(a);               \
            }                                                                                 \
        } else {                                                                              \
            if (md) {                                                                         \
                if (deg == 0) k_solve<DIMV, 0, MODE_MAP, double><<<b, 128, 0, s>>>(a);       \
                else if (deg == 1) k_solve<DIMV, 1, MODE_MAP, double><<<b, 128, 0, s>>>(a);  \
                else k_solve<DIMV, 2, MODE_MAP, double><<<b, 128, 0, s>>>(a);                \
            } else {                                                                          \
                if (deg == 0) k_solve<DIMV, 0, MODE_MAP, float><<<b, 128, 0, s>>>(a);        \
                else if (deg == 1) k_solve<DIMV, 1, MODE_MAP, float><<<b, 128, 0, s>>>(a);   \
                else k_solve<DIMV, 2, MODE_MAP, float><<<b, 128, 0, s>>>(a);                 \
            }                                                                                 \
        }                                                                                     \
        PCMS_LAUNCH_CHECK("k_solve");                                                         \
    }                                                                                         \
    void shape_dispatch_d##DIMV(int deg, bool mixed, int G, const ShapeArgs& a, int b,          \
                              cudaStream_t s) {                                               \
        if (G == 32) {                                                                        \
            if (mixed) {                                                                      \
                if (deg == 0) k_shape<DIMV, 0, true, 32><<<b, 256, 0, s>>>(a);               \
                else if (deg == 1) k_shape<DIMV, 1, true, 32><<<b, 256, 0, s>>>(a);          \
                else k_shape<DIMV, 2, true, 32><<<b, 256, 0, s>>>(a);                        \
            } else {                                                                          \
                if (deg == 0) k_shape<DIMV, 0, false, 32><<<b, 256, 0, s>>>(a);              \
                else if (deg == 1) k_shape<DIMV, 1, false, 32><<<b, 256, 0, s>>>(a);         \
                else k_shape<DIMV, 2, false, 32><<<b, 256, 0, s>>>(a);                       \
            }                                                                                 \
        } else {                                                                              \
            if (mixed) {                                                                      \
                if (deg == 0) k_shape<DIMV, 0, true, 8><<<b, 256, 0, s>>>(a);                \
                else if (deg == 1) k_shape<DIMV, 1, true, 8><<<b, 256, 0, s>>>(a);           \
                else k_shape<DIMV, 2, true, 8><<<b, 256, 0, s>>>(a);                         \
            } else {                                                                          \
                if (deg == 0) k_shape<DIMV, 0, false, 8><<<b, 256, 0, s>>>(a);               \
                else if (deg == 1) k_shape<DIMV, 1, false, 8><<<b, 256, 0, s>>>(a);          \
                else k_shape<DIMV, 2, false, 8><<<b, 256, 0, s>>>(a);                        \
            }                                                                                 \
        }                                                                                     \
        PCMS_LAUNCH_CHECK("k_shape");                                                         \
    }                                                                                         \
    template <int DEG>                                                                        \
    static void comp_mode(int mode, int G, const AsmArgs& a, int b, cudaStream_t s) {         \
        if (mode == MODE_MAP) {                                                               \
            if (G == 32) k_assemble<DIMV, DEG, true, MODE_MAP, 32, float, true><<<b, 256, 0, s>>>(a); \
            else k_assemble<DIMV, DEG, true, MODE_MAP, 8, float, true><<<b, 256, 0, s>>>(a);  \
        } else {                                                                              \
            if (G == 32) k_assemble<DIMV, DEG, true, MODE_FUSED, 32, float, true><<<b, 256, 0, s>>>(a); \
            else k_assemble<DIMV, DEG, true, MODE_FUSED, 8, float, true><<<b, 256, 0, s>>>(a); \
        }                                                                                     \
    }                                                                                         \
    void assemble_comp_dispatch_d##DIMV(int deg, int mode, int G, const AsmArgs& a, int b,    \
                                        cudaStream_t s) {                                     \
        if (deg == 0) comp_mode<0>(mode, G, a, b, s);                                         \
        else if (deg == 1) comp_mode<1>(mode, G, a, b, s);                                    \
        else comp_mode<2>(mode, G, a, b, s);                                                  \
        PCMS_LAUNCH_CHECK("k_assemble_comp");                                                 \
    }                                                                                         \
    }
