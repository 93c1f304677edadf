// mls_dispatch.cuh -- runtime dispatch of the templated MLS kernels. The definitions live
// in mls_inst_d2.cu / mls_inst_d3.cu so the two dimensions compile in parallel.
#pragma once

#include "mls_kernels.cuh"
#include "mls_map8.cuh"
#include "trace.cuh"

namespace pcms {

// assemble: mode MODE_COUNT / MODE_MAP / MODE_FUSED; G = lanes per target (8 or 32);
// field_double: FUSED field type (float or double)
#define PCMS_DECLARE_MLS_DISPATCH(DIMV)                                                       \
    void assemble_dispatch_d##DIMV(int deg, bool mixed, int mode, int G, int acc,             \
                                   bool field_double, const AsmArgs& a, int blocks,           \
                                   cudaStream_t s);                                           \
    void solve_dispatch_d##DIMV(int deg, int mode, int mom_kind, const SolveArgs& a,          \
                                int blocks, cudaStream_t s);                                  \
    void shape_dispatch_d##DIMV(int deg, bool mixed, int G, const ShapeArgs& a, int blocks,   \
                                cudaStream_t s);                                              \
    void shape_apply_dispatch_d##DIMV(int deg, int G, const ShapeArgs& a, int blocks,         \
                                      cudaStream_t s);
PCMS_DECLARE_MLS_DISPATCH(2)
PCMS_DECLARE_MLS_DISPATCH(3)

// stored moment types of the solve
enum { MOM_F32 = 0, MOM_F32PAIR = 1, MOM_F64 = 2 };

// acc: ACC_PLAIN, or ACC_BK (mixed MAP/FUSED: blocked compensation, float2 moments) for
// tier 1 of very large neighbourhoods (32 lanes) and for tier 2 (8 or 32 lanes, as tier 1).
inline void assemble_any(int dim, int deg, bool mixed, int mode, int G, int acc, bool fd,
                         const AsmArgs& a, int blocks, cudaStream_t s) {
    const bool bk = mixed && mode != MODE_COUNT && (G == 32 || G == 8) && acc == ACC_BK;
    // a target list means a later tier of the mixed path (tier 2: blocked FP32, tier 3: FP64)
    // or the FP64 path's refine pass (a list with a re-centred basis)
    static const char* names[6][3] = {
        {"mls_count_fp64", "mls_assemble_map_fp64", "mls_assemble_fused_fp64"},
        {"mls_count_mixed", "mls_assemble_map_mixed", "mls_assemble_fused_mixed"},
        {"mls_count_mixed", "mls_assemble_map_bk", "mls_assemble_fused_bk"},
        {"mls_count_mixed", "mls_assemble_map_tier2", "mls_assemble_fused_tier2"},
        {"mls_count_fp64", "mls_assemble_map_tier3", "mls_assemble_fused_tier3"},
        {"mls_count_fp64", "mls_assemble_map_fp64_refine", "mls_assemble_fused_fp64_refine"}};
    const int row = !mixed ? (a.list ? (a.basis ? 5 : 4) : 0) : (!bk ? 1 : (a.list ? 3 : 2));
    PCMS_TRACE(names[row][mode], s);
    if (dim == 2) assemble_dispatch_d2(deg, mixed, mode, G, bk ? ACC_BK : ACC_PLAIN, fd, a, blocks, s);
    else assemble_dispatch_d3(deg, mixed, mode, G, bk ? ACC_BK : ACC_PLAIN, fd, a, blocks, s);
}
inline void solve_any(int dim, int deg, int mode, int mom_kind, const SolveArgs& a, int blocks,
                      cudaStream_t s) {
    PCMS_TRACE(mode == MODE_FUSED ? "mls_solve_fused" : "mls_solve_map", s);
    if (dim == 2) solve_dispatch_d2(deg, mode, mom_kind, a, blocks, s);
    else solve_dispatch_d3(deg, mode, mom_kind, a, blocks, s);
}
inline void shape_any(int dim, int deg, bool mixed, int G, const ShapeArgs& a, int blocks,
                      cudaStream_t s) {
    PCMS_TRACE(mixed ? "mls_shape_mixed" : "mls_shape_fp64", s);
    if (dim == 2) shape_dispatch_d2(deg, mixed, G, a, blocks, s);
    else shape_dispatch_d3(deg, mixed, G, a, blocks, s);
}
// mixed rows evaluated and applied at once (a.fs, a.fp, a.status, a.stage), nothing stored
inline void shape_apply_any(int dim, int deg, int G, const ShapeArgs& a, int blocks,
                            cudaStream_t s) {
    PCMS_TRACE("mls_shape_apply_mixed", s);
    if (dim == 2) shape_apply_dispatch_d2(deg, G, a, blocks, s);
    else shape_apply_dispatch_d3(deg, G, a, blocks, s);
}

}  // namespace pcms

// Definitions for one dimension; included by exactly one .cu per dimension.
#define PCMS_DEFINE_MLS_DISPATCH(DIMV)                                                        \
    namespace pcms {                                                                          \
    template <int DEG, bool MIXED>                                                            \
    static void asm_mode(int mode, int G, int acc, bool fd, const AsmArgs& a, int b,          \
                         cudaStream_t s) {                                                    \
        if (mode == MODE_COUNT) {                                                             \
            if (DEG != 0) return;                                                             \
            if (G == 32) k_assemble<DIMV, 0, MIXED, MODE_COUNT, 32, float><<<b, 256, 0, s>>>(a); \
            else k_assemble<DIMV, 0, MIXED, MODE_COUNT, 8, float><<<b, 256, 0, s>>>(a);       \
        } else if (mode == MODE_MAP) {                                                        \
            if (G == 32 && MIXED && acc == ACC_BK)                                            \
                k_assemble<DIMV, DEG, MIXED, MODE_MAP, 32, float, MIXED ? ACC_BK : ACC_PLAIN><<<b, 256, 0, s>>>(a); \
            else if (MIXED && acc == ACC_BK)                                                  \
                k_assemble<DIMV, DEG, MIXED, MODE_MAP, 8, float, MIXED ? ACC_BK : ACC_PLAIN><<<b, 256, 0, s>>>(a); \
            else if (G == 32) k_assemble<DIMV, DEG, MIXED, MODE_MAP, 32, float><<<b, 256, 0, s>>>(a); \
            else launch_map8<DIMV, DEG, MIXED>(a, b, s);                                       \
        } else {                                                                              \
            if (fd) {                                                                         \
                if constexpr (!MIXED) {                                                       \
                    if (G == 32) k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 32, double><<<b, 256, 0, s>>>(a); \
                    else k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 8, double><<<b, 256, 0, s>>>(a); \
                }                                                                             \
            } else {                                                                          \
                if (G == 32 && MIXED && acc == ACC_BK)                                        \
                    k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 32, float, MIXED ? ACC_BK : ACC_PLAIN><<<b, 256, 0, s>>>(a); \
                else if (MIXED && acc == ACC_BK)                                              \
                    k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 8, float, MIXED ? ACC_BK : ACC_PLAIN><<<b, 256, 0, s>>>(a); \
                else if (G == 32) k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 32, float><<<b, 256, 0, s>>>(a); \
                else k_assemble<DIMV, DEG, MIXED, MODE_FUSED, 8, float><<<b, 256, 0, s>>>(a);  \
            }                                                                                 \
        }                                                                                     \
    }                                                                                         \
    void assemble_dispatch_d##DIMV(int deg, bool mixed, int mode, int G, int acc, bool fd,      \
                                 const AsmArgs& a, int b, cudaStream_t s) {                   \
        if (mode == MODE_COUNT) deg = 0;                                                      \
        if (mixed) {                                                                          \
            if (deg == 0) asm_mode<0, true>(mode, G, acc, fd, a, b, s);                       \
            else if (deg == 1) asm_mode<1, true>(mode, G, acc, fd, a, b, s);                  \
            else asm_mode<2, true>(mode, G, acc, fd, a, b, s);                                \
        } else {                                                                              \
            if (deg == 0) asm_mode<0, false>(mode, G, acc, fd, a, b, s);                      \
            else if (deg == 1) asm_mode<1, false>(mode, G, acc, fd, a, b, s);                 \
            else asm_mode<2, false>(mode, G, acc, fd, a, b, s);                               \
        }                                                                                     \
        PCMS_LAUNCH_CHECK("k_assemble");                                                      \
    }                                                                                         \
    template <int DEG, int MODE>                                                              \
    static void solve_deg(int mk, const SolveArgs& a, int b, cudaStream_t s) {                \
        if (mk == MOM_F64) {                                                                  \
            k_solve<DIMV, DEG, MODE, double><<<b, 128, 0, s>>>(a);                            \
        } else if (mk == MOM_F32PAIR) {                                                       \
            k_solve<DIMV, DEG, MODE, float2, 1><<<b, 128, 0, s>>>(a);                         \
            k_solve<DIMV, DEG, MODE, float2, 2><<<b, 128, 0, s>>>(a);                         \
        } else {                                                                              \
            k_solve<DIMV, DEG, MODE, float, 1><<<b, 128, 0, s>>>(a);                          \
            k_solve<DIMV, DEG, MODE, float, 2><<<b, 128, 0, s>>>(a);                          \
        }                                                                                     \
    }                                                                                         \
    void solve_dispatch_d##DIMV(int deg, int mode, int mk, const SolveArgs& a, int b,           \
                              cudaStream_t s) {                                               \
        if (mode == MODE_FUSED) {                                                             \
            if (deg == 0) solve_deg<0, MODE_FUSED>(mk, a, b, s);                              \
            else if (deg == 1) solve_deg<1, MODE_FUSED>(mk, a, b, s);                         \
            else solve_deg<2, MODE_FUSED>(mk, a, b, s);                                       \
        } else {                                                                              \
            if (deg == 0) solve_deg<0, MODE_MAP>(mk, a, b, s);                                \
            else if (deg == 1) solve_deg<1, MODE_MAP>(mk, a, b, s);                           \
            else solve_deg<2, MODE_MAP>(mk, a, b, s);                                         \
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
    void shape_apply_dispatch_d##DIMV(int deg, int G, const ShapeArgs& a, int b,              \
                                      cudaStream_t s) {                                       \
        if (G == 32) {                                                                        \
            if (deg == 0) k_shape<DIMV, 0, true, 32, true><<<b, 256, 0, s>>>(a);             \
            else if (deg == 1) k_shape<DIMV, 1, true, 32, true><<<b, 256, 0, s>>>(a);        \
            else k_shape<DIMV, 2, true, 32, true><<<b, 256, 0, s>>>(a);                      \
        } else {                                                                              \
            if (deg == 0) k_shape<DIMV, 0, true, 8, true><<<b, 256, 0, s>>>(a);              \
            else if (deg == 1) k_shape<DIMV, 1, true, 8, true><<<b, 256, 0, s>>>(a);         \
            else k_shape<DIMV, 2, true, 8, true><<<b, 256, 0, s>>>(a);                       \
        }                                                                                     \
        PCMS_LAUNCH_CHECK("k_shape_apply");                                                   \
    }                                                                                         \
    }
