// Per-problem kernels: the merged-form step of one context (state y, or the
// rotated basis z = T^T y of MLN_FORM_ROTATED) written out as
// straight-line code with the constants as literals and the exactly-zero
// entries of the set-up matrices left out, compiled at run time for sm_103a
// (NVRTC) and launched through the driver API. In the merged form the
// arithmetic and its order are those of the register cell model, so the
// results are bit-identical; the kernel just skips multiplications by zero and
// needs no constant-bank loads. The rotated form exists only here.
//
// NVRTC and the driver entry points are looked up at run time (dlopen and
// cudaGetDriverEntryPointByVersion): without them the JIT model is reported
// unavailable and the other cell models still work.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "dispatch.cuh"
#include "jit.h"
#include "setup.h"

#include "jit_source.inc"

namespace mln {
namespace {

// ---- NVRTC, loaded on first use
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram *nvrtcProgram_t;
struct Nvrtc {
    nvrtcResult_t (*create)(nvrtcProgram_t *, const char *, const char *, int, const char *const *,
                            const char *const *) = nullptr;
    nvrtcResult_t (*compile)(nvrtcProgram_t, int, const char *const *) = nullptr;
    nvrtcResult_t (*log_size)(nvrtcProgram_t, size_t *) = nullptr;
    nvrtcResult_t (*log)(nvrtcProgram_t, char *) = nullptr;
    nvrtcResult_t (*cubin_size)(nvrtcProgram_t, size_t *) = nullptr;
    nvrtcResult_t (*cubin)(nvrtcProgram_t, char *) = nullptr;
    nvrtcResult_t (*destroy)(nvrtcProgram_t *) = nullptr;
    bool ok = false;
};

// ---- driver API, through the runtime's entry-point query
struct Driver {
    CUresult (*load)(CUmodule *, const void *) = nullptr;
    CUresult (*get)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                       void **, void **) = nullptr;
    CUresult (*set_attr)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*launch_ex)(const CUlaunchConfig *, CUfunction, void **, void **) = nullptr;  // optional
    bool ok = false;
};

std::mutex g_mu;
Nvrtc g_nvrtc;
Driver g_drv;
bool g_tried = false;
std::string g_why;
std::map<std::pair<int, std::string>, CUmodule> g_cache;  // (device, source) -> loaded module

template <typename F>
bool sym(void *h, const char *name, F &f) {
    f = reinterpret_cast<F>(dlsym(h, name));
    return f != nullptr;
}

template <typename F>
bool entry(const char *name, F &f) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    f = reinterpret_cast<F>(p);
    return true;
}

bool load_tools() {
    if (g_tried) return g_nvrtc.ok && g_drv.ok;
    g_tried = true;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *n : names)
        if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
        g_why = "libnvrtc not found";
        return false;
    }
    Nvrtc &r = g_nvrtc;
    r.ok = sym(h, "nvrtcCreateProgram", r.create) && sym(h, "nvrtcCompileProgram", r.compile) &&
           sym(h, "nvrtcGetProgramLogSize", r.log_size) && sym(h, "nvrtcGetProgramLog", r.log) &&
           sym(h, "nvrtcGetCUBINSize", r.cubin_size) && sym(h, "nvrtcGetCUBIN", r.cubin) &&
           sym(h, "nvrtcDestroyProgram", r.destroy);
    Driver &d = g_drv;
    d.ok = entry("cuModuleLoadData", d.load) && entry("cuModuleGetFunction", d.get) &&
           entry("cuLaunchKernel", d.launch) && entry("cuFuncSetAttribute", d.set_attr);
    if (!entry("cuLaunchKernelEx", d.launch_ex)) d.launch_ex = nullptr;
    if (!r.ok) g_why = "NVRTC symbols missing";
    else if (!d.ok) g_why = "driver entry points unavailable";
    return r.ok && d.ok;
}

std::string lit(double v, bool fp32) {
    char buf[64];
    if (fp32) std::snprintf(buf, sizeof(buf), "%af", static_cast<double>(static_cast<float>(v)));
    else std::snprintf(buf, sizeof(buf), "%a", v);
    return buf;
}

bool nz(double v, bool fp32) { return fp32 ? static_cast<float>(v) != 0.0f : v != 0.0; }

// sum_j A[i][j] x_j over the non-zero entries, in column order, as the dense
// product does: first term a product, then fused multiply-adds onto it.
std::string row_sum(const std::vector<double> &A, int ld, int i, int ncols, const std::string &x, bool fp32,
                    const std::string &init = "") {
    std::string acc = init;
    for (int j = 0; j < ncols; ++j) {
        double a = A[i * ld + j];
        if (!nz(a, fp32)) continue;
        std::string t = x + "[" + std::to_string(j) + "]";
        // the first product is rounded on its own (as in the dense chain, where
        // fused multiply-adds follow it), never contracted into a later add
        if (acc.empty()) acc = std::string(fp32 ? "__fmul_rn(" : "__dmul_rn(") + lit(a, fp32) + ", " + t + ")";
        else acc = "fma(" + lit(a, fp32) + ", " + t + ", " + acc + ")";
    }
    return acc;
}

}  // namespace

unsigned jit_body_flags(const mln_params &p) {
    return (p.boundary == MLN_BC_PERIODIC ? kBodyRing : kBodyOpen) |
           (p.source_kind == MLN_SRC_NONE ? kBodyNoSrc : 0u) | kBodyNoRec;
}

std::string jit_merged_source(const Setup &s, double dt, bool fp32, bool rotated, unsigned body_flags) {
    const int N = s.N, D = s.D, Q = s.q, P = 2 * Q;
    const char *R = fp32 ? "float" : "double";
    std::ostringstream o;
    o << "#define MLN_JIT 1\n"
      << "#ifdef __CUDACC_RTC__\ntypedef long long int64_t;\ntypedef int int32_t;\n#endif\n"
      << kKernelsSource << "\nnamespace mln {\n"
      << "struct JitConsts { int unused; };\n"
      << "struct JitCell {\n  static constexpr int D = " << D << ";\n  using Consts = JitConsts;\n  " << R
      << " s[D];\n"
      << "  __device__ __forceinline__ void setup(unsigned char *, const Consts &) {}\n"
      << "  __device__ __forceinline__ void load(const " << R
      << " *src, int64_t stride, int64_t m) { for (int i = 0; i < D; ++i) s[i] = src[i * stride + m]; }\n"
      << "  __device__ __forceinline__ void store(" << R
      << " *dst, int64_t stride, int64_t m) const { for (int i = 0; i < D; ++i) dst[i * stride + m] = s[i]; }\n"
      << "  __device__ __forceinline__ void end_step() {}\n"
      << "  __device__ __forceinline__ " << R << " step(" << R << " e, const Consts &) {\n"
      << "    " << R << " z[D], y[D];\n";
    // z = T^T y on the plane rows (T^T row k = T column k); in the rotated
    // form the state already is z
    std::vector<double> Tt((size_t)D * D);
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) Tt[k * D + i] = s.T[i * D + k];
    for (int k = 0; k < P; ++k) {
        std::string e = rotated ? "s[" + std::to_string(k) + "]" : row_sum(Tt, D, k, D, "s", fp32);
        o << "    z[" << k << "] = " << (e.empty() ? std::string(fp32 ? "0.0f" : "0.0") : e) << ";\n";
    }
    for (int k = P; k < D; ++k) o << "    z[" << k << "] = " << (fp32 ? "0.0f" : "0.0") << ";\n";
    o << "    const " << R << " psi[" << (N - 1) << "] = {";
    for (int a = 0; a < N - 1; ++a) o << (a ? ", " : "") << lit(s.psi[a] * dt, fp32);
    o << "};\n    rotation_increment<" << N << ">(z, psi, e);\n";
    // y'' = y + T (R - I) z on the plane columns: accumulated onto y in FP64,
    // the increment summed first in FP32 (as the register model)
    for (int i = 0; i < D; ++i) {
        const std::string si = "s[" + std::to_string(i) + "]";
        if (rotated) {  // z'' = z + (R - I) z on the plane pairs, the rest unchanged
            o << "    y[" << i << "] = " << (i < P ? si + " + z[" + std::to_string(i) + "]" : si) << ";\n";
        } else if (fp32) {
            std::string e = row_sum(s.T, D, i, P, "z", fp32);
            o << "    y[" << i << "] = " << (e.empty() ? si : si + " + (" + e + ")") << ";\n";
        } else {
            o << "    y[" << i << "] = " << row_sum(s.T, D, i, P, "z", fp32, si) << ";\n";
        }
    }
    // dP/dt = wm . y'' + cm (rotated: wz . z'' + cm)
    const std::vector<double> &wv = rotated ? s.wz : s.wm;
    const std::vector<double> &Cm = rotated ? s.C1z : s.C1;
    const std::vector<double> &bv = rotated ? s.cz : s.b2;
    {
        std::string acc = lit(s.cm, fp32);
        for (int i = 0; i < D; ++i)
            if (nz(wv[i], fp32)) acc = "fma(" + lit(wv[i], fp32) + ", y[" + std::to_string(i) + "], " + acc + ")";
        o << "    const " << R << " dpdt = " << acc << ";\n";
    }
    // y = (y'' + b2) + C1 y'' accumulated onto y'' + b2 (no add where b2 is
    // zero) in FP64; y'' + (C1 y'' + b2) in FP32
    for (int i = 0; i < D; ++i) {
        const std::string yi = "y[" + std::to_string(i) + "]";
        if (fp32) {
            std::string e = row_sum(Cm, D, i, D, "y", fp32, lit(bv[i], fp32));
            o << "    s[" << i << "] = " << yi << " + (" << e << ");\n";
        } else {
            const std::string init = nz(bv[i], fp32) ? "(" + yi + " + " + lit(bv[i], fp32) + ")" : yi;
            o << "    s[" << i << "] = " << row_sum(Cm, D, i, D, "y", fp32, init) << ";\n";
        }
    }
    o << "    return dpdt;\n  }\n};\n"
      << "extern \"C\" __global__ void __launch_bounds__(kMaxThreads, 1) mln_jit_step(const __grid_constant__ BlockArgs<"
      << R << "> a, const __grid_constant__ JitConsts k) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      // launched with a programmatic dependency on the kernel before it:
      // wait for that grid to complete (its fields and states visible) before
      // any read or write, then let the next launch be placed
      << "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
      << "  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n"
      << "  block_body<" << N << ", " << R << ", JitCell, " << body_flags
      << "u>(a, k, static_cast<int64_t>(blockIdx.x), smem_raw);\n}\n"
      << "}  // namespace mln\n";
    return o.str();
}

namespace {

// A double constant as the FP32 pair (hi, lo) of double-float arithmetic.
struct DfLit {
    std::string h, l;
    bool has_l;
};
DfLit df_lit(double v) {
    const float h = static_cast<float>(v);
    const float l = static_cast<float>(v - static_cast<double>(h));
    return {lit(h, true), lit(l, true), l != 0.0f};
}

// dst = init (+ c) + sum_j A[i][j] x_j in double-float: the high words summed
// exactly, every rounding error in the low word, normalised at the end.
void df_row(std::ostringstream &o, const std::vector<double> &A, int ld, int i, int ncols, const std::string &x,
            const std::string &dst, const std::string &init, double c = 0.0) {
    o << "    { float ah = 0.0f, al = 0.0f;";
    bool started = false;
    if (!init.empty()) {
        o << " ah = " << init << ".h; al = " << init << ".l;";
        started = true;
    }
    if (c != 0.0) {
        const DfLit k = df_lit(c);
        if (started) o << " df_add(ah, al, " << k.h << ", " << k.l << ");";
        else o << " ah = " << k.h << "; al = " << k.l << ";";
        started = true;
    }
    for (int j = 0; j < ncols; ++j) {
        const double a = A[i * ld + j];
        if (a == 0.0) continue;
        const DfLit k = df_lit(a);
        const std::string t = x + "[" + std::to_string(j) + "]";
        o << "\n      ";
        if (!started) {
            if (k.has_l) o << "df_first(ah, al, " << k.h << ", " << k.l << ", " << t << ");";
            else o << "df_first1(ah, al, " << k.h << ", " << t << ");";
            started = true;
        } else {
            if (k.has_l) o << "df_acc(ah, al, " << k.h << ", " << k.l << ", " << t << ");";
            else o << "df_acc1(ah, al, " << k.h << ", " << t << ");";
        }
    }
    o << "\n      " << dst << " = df_norm(ah, al); }\n";
}

}  // namespace

int df_threads(int D, bool rotated) { return rotated && D > 15 ? 256 : kMaxThreads; }

bool df_constants_in_range(const Setup &s, double dt, bool rotated) {
    auto ok = [](double v) { return v == 0.0 || (std::fabs(v) < 1e37 && std::fabs(v) > 1e-30); };
    const int D = s.D, P = 2 * s.q;
    const std::vector<double> &Cm = rotated ? s.C1z : s.C1, &wv = rotated ? s.wz : s.wm, &bv = rotated ? s.cz : s.b2;
    for (int i = 0; i < D; ++i) {
        if (!rotated)
            for (int k = 0; k < P; ++k)
                if (!ok(s.T[i * D + k])) return false;
        for (int j = 0; j < D; ++j)
            if (!ok(Cm[i * D + j])) return false;
        if (!ok(wv[i]) || !ok(bv[i])) return false;
    }
    for (int a = 0; a < s.N - 1; ++a)
        if (!ok(s.psi[a] * dt)) return false;
    return ok(s.cm);
}

std::string jit_df_source(const Setup &s, double dt, unsigned body_flags, bool rotated) {
    const int N = s.N, D = s.D, Q = s.q, P = 2 * Q;
    const std::vector<double> &Cm = rotated ? s.C1z : s.C1, &wv = rotated ? s.wz : s.wm, &bv = rotated ? s.cz : s.b2;
    std::ostringstream o;
    o << "#define MLN_JIT 1\n"
      << "#ifdef __CUDACC_RTC__\ntypedef long long int64_t;\ntypedef int int32_t;\n#endif\n"
      << kKernelsSource << "\nnamespace mln {\n"
      << "struct JitConsts { int unused; };\n"
      << "// the merged step in double-float arithmetic, E, H and dP/dt as pairs too;\n"
      << "// the state, E and H in FP64 memory, converted at the ends of a launch\n"
      << "struct JitCell {\n  static constexpr int D = " << D << ";\n  using Consts = JitConsts;\n"
      << "  using Field = Df;\n  Df s[D];\n"
      << "  __device__ __forceinline__ void setup(unsigned char *, const Consts &) {}\n"
      << "  __device__ __forceinline__ void load(const double *src, int64_t stride, int64_t m) { for (int i = 0; i < D; "
         "++i) s[i] = df_of(src[i * stride + m]); }\n"
      << "  __device__ __forceinline__ void store(double *dst, int64_t stride, int64_t m) const { for (int i = 0; i < "
         "D; ++i) dst[i * stride + m] = df_value(s[i]); }\n"
      << "  __device__ __forceinline__ void end_step() {}\n"
      << "  __device__ __forceinline__ Df step(Df e, const Consts &) {\n"
      << "    Df z[D], y[D];\n";
    // z = T^T y on the plane rows; in the rotated form the state already is z
    std::vector<double> Tt((size_t)D * D);
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) Tt[k * D + i] = s.T[i * D + k];
    for (int k = 0; k < P; ++k) {
        if (rotated) o << "    z[" << k << "] = s[" << k << "];\n";
        else df_row(o, Tt, D, k, D, "s", "z[" + std::to_string(k) + "]", "");
    }
    for (int k = P; k < D; ++k) o << "    z[" << k << "] = Df{0.0f, 0.0f};\n";
    o << "    const float psi_h[" << (N - 1) << "] = {";
    for (int a = 0; a < N - 1; ++a) o << (a ? ", " : "") << df_lit(s.psi[a] * dt).h;
    o << "}, psi_l[" << (N - 1) << "] = {";
    for (int a = 0; a < N - 1; ++a) o << (a ? ", " : "") << df_lit(s.psi[a] * dt).l;
    o << "};\n    df_rotation_increment<" << N << ">(z, psi_h, psi_l, e);\n";
    // y'' = y + T (R - I) z on the plane columns; rotated: z'' = z + (R - I) z
    // on the plane pairs, the rest unchanged
    for (int i = 0; i < D; ++i) {
        const std::string si = "s[" + std::to_string(i) + "]", yi = "y[" + std::to_string(i) + "]";
        if (!rotated)
            df_row(o, s.T, D, i, P, "z", yi, si);
        else if (i < P)
            o << "    { float ah = " << si << ".h, al = " << si << ".l; df_add(ah, al, z[" << i << "].h, z[" << i
              << "].l); " << yi << " = df_norm(ah, al); }\n";
        else
            o << "    " << yi << " = " << si << ";\n";
    }
    // dP/dt = cm + wm . y'' (rotated: wz . z'')
    {
        const DfLit k = df_lit(s.cm);
        o << "    Df dpdt;\n    { float ah = " << k.h << ", al = " << k.l << ";";
        for (int i = 0; i < D; ++i) {
            if (wv[i] == 0.0) continue;
            const DfLit w = df_lit(wv[i]);
            o << "\n      " << (w.has_l ? "df_acc(ah, al, " + w.h + ", " + w.l : "df_acc1(ah, al, " + w.h) << ", y["
              << i << "]);";
        }
        o << "\n      dpdt = df_norm(ah, al); }\n";
    }
    // y = (y'' + b2) + C1 y'' (rotated: z = (z'' + c') + C1z z'')
    for (int i = 0; i < D; ++i)
        df_row(o, Cm, D, i, D, "y", "s[" + std::to_string(i) + "]", "y[" + std::to_string(i) + "]", bv[i]);
    o << "    return dpdt;\n  }\n};\n"
      << "extern \"C\" __global__ void __launch_bounds__(" << (df_threads(D, rotated) == kMaxThreads ? "kMaxThreads" : "256")
      << ", 1) mln_jit_step(const __grid_constant__ "
         "BlockArgs<double> a, const __grid_constant__ JitConsts k) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
      << "  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n"
      << "  block_body<" << N << ", double, JitCell, " << body_flags
      << "u>(a, k, static_cast<int64_t>(blockIdx.x), smem_raw);\n}\n"
      << "}  // namespace mln\n";
    return o.str();
}

void batch_pattern_add(BatchPattern &pat, const Setup &s, const mln_params &p, bool fp32) {
    const int D = s.D, P = 2 * s.q;
    pat.flags &= jit_body_flags(p);
    if (pat.N == 0) {
        pat.N = s.N;
        pat.tt.assign(static_cast<size_t>(P) * D, 0);
        pat.t.assign(static_cast<size_t>(D) * P, 0);
        pat.wm.assign(D, 0);
        pat.c1.assign(static_cast<size_t>(D) * D, 0);
    }
    for (int k = 0; k < P; ++k)
        for (int i = 0; i < D; ++i) pat.tt[k * D + i] |= nz(s.T[i * D + k], fp32);
    for (int i = 0; i < D; ++i)
        for (int p = 0; p < P; ++p) pat.t[i * P + p] |= nz(s.T[i * D + p], fp32);
    for (int i = 0; i < D; ++i) pat.wm[i] |= nz(s.wm[i], fp32);
    for (int i = 0; i < D * D; ++i) pat.c1[i] |= nz(s.C1[i], fp32);
}

// The distinct constants of the batched step, in a fixed order: the entries
// of T in the pattern (plane columns, row by row: each is used twice, by
// T^T y and by T dz), psi dt, c', wm, then per row of C1: b2_i and the
// row's entries. f(value) for each; the index of a constant is its position.
template <typename F>
void batch_walk(const BatchPattern &pat, const Setup *s, double dt, F f) {
    const int N = pat.N, D = N * N - 1, P = N * (N - 1);
    for (int i = 0; i < D; ++i)
        for (int p = 0; p < P; ++p)
            if (pat.t[i * P + p] || pat.tt[p * D + i]) f(s ? s->T[i * D + p] : 0.0);
    for (int a = 0; a < N - 1; ++a) f(s ? s->psi[a] * dt : 0.0);
    f(s ? s->cm : 0.0);
    for (int i = 0; i < D; ++i)
        if (pat.wm[i]) f(s ? s->wm[i] : 0.0);
    for (int i = 0; i < D; ++i) {
        f(s ? s->b2[i] : 0.0);
        for (int j = 0; j < D; ++j)
            if (pat.c1[i * D + j]) f(s ? s->C1[i * D + j] : 0.0);
    }
}

int batch_consts_count(const BatchPattern &pat) {
    int n = 0;
    batch_walk(pat, nullptr, 0.0, [&](double) { ++n; });
    return n;
}

void batch_pack(const BatchPattern &pat, const Setup &s, double dt, bool fp32, std::vector<unsigned char> &out,
                bool df) {
    out.clear();
    batch_walk(pat, &s, dt, [&](double x) {
        if (df) {  // the (hi, lo) FP32 pair of the double
            const float f[2] = {static_cast<float>(x), static_cast<float>(x - static_cast<double>(static_cast<float>(x)))};
            const unsigned char *b = reinterpret_cast<const unsigned char *>(f);
            out.insert(out.end(), b, b + 8);
        } else if (fp32) {
            const float f = static_cast<float>(x);
            const unsigned char *b = reinterpret_cast<const unsigned char *>(&f);
            out.insert(out.end(), b, b + 4);
        } else {
            const unsigned char *b = reinterpret_cast<const unsigned char *>(&x);
            out.insert(out.end(), b, b + 8);
        }
    });
    out.resize((out.size() + 15) / 16 * 16, 0);
}

std::string jit_batch_df_source(const BatchPattern &pat);

std::string jit_batch_source(const BatchPattern &pat, bool fp32, bool df) {
    if (df) return jit_batch_df_source(pat);
    const int N = pat.N, D = N * N - 1, P = N * (N - 1);
    const char *R = fp32 ? "float" : "double";
    const int nc = batch_consts_count(pat);
    const int words = nc * (fp32 ? 1 : 2);
    // constants in registers (read from shared memory once per launch) when
    // they fit next to the state; else read from shared memory at each use
    const bool regs = words <= 176;
    const int ncp = (nc * (fp32 ? 4 : 8) + 15) / 16 * 16 / (fp32 ? 4 : 8);
    // index of each distinct constant (the order of batch_walk)
    std::vector<int> iT(static_cast<size_t>(D) * P, -1), iW(D, -1), iB(D, -1), iC(static_cast<size_t>(D) * D, -1);
    std::vector<int> iPsi(N - 1);
    int idx = 0, iCm = -1;
    for (int i = 0; i < D; ++i)
        for (int p = 0; p < P; ++p)
            if (pat.t[i * P + p] || pat.tt[p * D + i]) iT[i * P + p] = idx++;
    for (int a = 0; a < N - 1; ++a) iPsi[a] = idx++;
    iCm = idx++;
    for (int i = 0; i < D; ++i)
        if (pat.wm[i]) iW[i] = idx++;
    for (int i = 0; i < D; ++i) {
        iB[i] = idx++;
        for (int j = 0; j < D; ++j)
            if (pat.c1[i * D + j]) iC[i * D + j] = idx++;
    }
    auto C = [&](int k) { return std::string(regs ? "c[" : "k.c[") + std::to_string(k) + "]"; };
    std::ostringstream o;
    o << "#define MLN_JIT 1\n"
      << "#ifdef __CUDACC_RTC__\ntypedef long long int64_t;\ntypedef int int32_t;\ntypedef unsigned int uint32_t;\n#endif\n"
      << kKernelsSource << "\nnamespace mln {\n"
      << "struct JitBatchConsts { " << R << " c[" << ncp << "]; };\n"
      << "struct JitBatchCell {\n  static constexpr int D = " << D << ";\n  using Consts = JitBatchConsts;\n  " << R
      << " s[D];\n";
    if (regs) o << "  " << R << " c[" << nc << "];\n";
    o << "  __device__ __forceinline__ void setup(unsigned char *, const Consts &k) {";
    if (regs) o << " for (int i = 0; i < " << nc << "; ++i) c[i] = k.c[i];";
    o << " }\n"
      << "  __device__ __forceinline__ void load(const " << R
      << " *src, int64_t stride, int64_t m) { for (int i = 0; i < D; ++i) s[i] = src[i * stride + m]; }\n"
      << "  __device__ __forceinline__ void load_cg(const " << R
      << " *src, int64_t stride, int64_t m) { for (int i = 0; i < D; ++i) s[i] = __ldcg(src + i * stride + m); }\n"
      << "  __device__ __forceinline__ void store(" << R
      << " *dst, int64_t stride, int64_t m) const { for (int i = 0; i < D; ++i) dst[i * stride + m] = s[i]; }\n"
      << "  __device__ __forceinline__ void end_step() {}\n"
      << "  __device__ __forceinline__ " << R << " step(" << R << " e, const Consts &k) {\n"
      << "    " << R << " z[D], y[D];\n";
    const std::string mul = fp32 ? "__fmul_rn(" : "__dmul_rn(";
    const std::string zero = fp32 ? "0.0f" : "0.0";
    // z = T^T y on the plane rows (T^T row k = T column k)
    for (int k = 0; k < P; ++k) {
        std::string acc;
        for (int i = 0; i < D; ++i) {
            if (!pat.tt[k * D + i]) continue;
            const std::string t = "s[" + std::to_string(i) + "]", c = C(iT[i * P + k]);
            acc = acc.empty() ? mul + c + ", " + t + ")" : "fma(" + c + ", " + t + ", " + acc + ")";
        }
        o << "    z[" << k << "] = " << (acc.empty() ? zero : acc) << ";\n";
    }
    for (int k = P; k < D; ++k) o << "    z[" << k << "] = " << zero << ";\n";
    o << "    const " << R << " psi[" << (N - 1) << "] = {";
    for (int a = 0; a < N - 1; ++a) o << (a ? ", " : "") << C(iPsi[a]);
    o << "};\n    rotation_increment<" << N << ">(z, psi, e);\n";
    // y'' = y + T (R - I) z on the plane columns (onto y in FP64, as the register model)
    for (int i = 0; i < D; ++i) {
        const std::string si = "s[" + std::to_string(i) + "]";
        std::string acc = fp32 ? "" : si;
        for (int p = 0; p < P; ++p) {
            if (!pat.t[i * P + p]) continue;
            const std::string t = "z[" + std::to_string(p) + "]", c = C(iT[i * P + p]);
            acc = acc.empty() ? mul + c + ", " + t + ")" : "fma(" + c + ", " + t + ", " + acc + ")";
        }
        if (fp32) acc = acc.empty() ? si : si + " + (" + acc + ")";
        o << "    y[" << i << "] = " << acc << ";\n";
    }
    // dP/dt = wm . y'' + c'
    {
        std::string acc = C(iCm);
        for (int i = 0; i < D; ++i)
            if (pat.wm[i]) acc = "fma(" + C(iW[i]) + ", y[" + std::to_string(i) + "], " + acc + ")";
        o << "    const " << R << " dpdt = " << acc << ";\n";
    }
    // y = (y'' + b2) + C1 y'' onto y'' + b2 in FP64; y'' + (C1 y'' + b2) in FP32
    for (int i = 0; i < D; ++i) {
        const std::string yi = "y[" + std::to_string(i) + "]";
        std::string acc = fp32 ? C(iB[i]) : "(" + yi + " + " + C(iB[i]) + ")";
        for (int j = 0; j < D; ++j)
            if (pat.c1[i * D + j]) acc = "fma(" + C(iC[i * D + j]) + ", y[" + std::to_string(j) + "], " + acc + ")";
        o << "    s[" << i << "] = " << (fp32 ? yi + " + (" + acc + ")" : acc) << ";\n";
    }
    o << "    return dpdt;\n  }\n};\n"
      << "extern \"C\" __global__ void __launch_bounds__(kBatchThreads, 1) mln_jit_batch(const BatchGrid<" << R
      << "> *grids, const BatchItem *items, const unsigned char *consts, int parity, int nsteps, int halo, int tile, "
         "int64_t step_offset) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  batch_body<" << N << ", " << R << ", JitBatchCell, " << (pat.flags == ~0u ? 0u : pat.flags)
      << "u>(grids, items, consts, parity, nsteps, halo, tile, step_offset, smem_raw);\n}\n"
      // every chunk of a call in one persistent launch (see batch_persistent)
      << "extern \"C\" __global__ void __launch_bounds__(kBatchThreads, 1) mln_jit_batch_persist(const BatchGrid<" << R
      << "> *grids, const BatchItem *items, const unsigned char *consts, int halo, int tile, int64_t step_offset, "
         "BatchPersist p) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  batch_persistent<" << N << ", " << R << ", JitBatchCell, " << (pat.flags == ~0u ? 0u : pat.flags)
      << "u>(grids, items, consts, halo, tile, step_offset, p, smem_raw);\n}\n"
      << "}  // namespace mln\n";
    return o.str();
}

// The batched step of the FP64 grids of one N in double-float pairs (the
// step of jit_df_source with each grid's constants as (hi, lo) pairs staged
// by batch_pack, over the union pattern: a term whose constant is zero for a
// grid leaves that grid's pair sums unchanged).
std::string jit_batch_df_source(const BatchPattern &pat) {
    const int N = pat.N, D = N * N - 1, P = N * (N - 1);
    const int nc = batch_consts_count(pat);
    const bool regs = 2 * nc <= 176;  // pairs in registers, as FP64 words
    const int ncp = (nc * 8 + 15) / 16 * 16 / 8;
    std::vector<int> iT(static_cast<size_t>(D) * P, -1), iW(D, -1), iB(D, -1), iC(static_cast<size_t>(D) * D, -1);
    std::vector<int> iPsi(N - 1);
    int idx = 0, iCm = -1;
    for (int i = 0; i < D; ++i)
        for (int p = 0; p < P; ++p)
            if (pat.t[i * P + p] || pat.tt[p * D + i]) iT[i * P + p] = idx++;
    for (int a = 0; a < N - 1; ++a) iPsi[a] = idx++;
    iCm = idx++;
    for (int i = 0; i < D; ++i)
        if (pat.wm[i]) iW[i] = idx++;
    for (int i = 0; i < D; ++i) {
        iB[i] = idx++;
        for (int j = 0; j < D; ++j)
            if (pat.c1[i * D + j]) iC[i * D + j] = idx++;
    }
    auto C = [&](int k) { return std::string(regs ? "c[" : "k.c[") + std::to_string(k) + "]"; };
    // dst = init (+ b) + sum of the pattern's terms, normalised once
    auto row = [&](std::ostringstream &o, const std::string &dst, const std::string &init, int ib,
                   const std::vector<std::pair<int, std::string>> &terms) {
        o << "    { float ah = 0.0f, al = 0.0f;";
        bool started = false;
        if (!init.empty()) {
            o << " ah = " << init << ".h; al = " << init << ".l;";
            started = true;
        }
        if (ib >= 0) {
            o << (started ? " df_add(ah, al, " + C(ib) + ".h, " + C(ib) + ".l);"
                          : " ah = " + C(ib) + ".h; al = " + C(ib) + ".l;");
            started = true;
        }
        for (const auto &t : terms) {
            o << "\n      " << (started ? "df_acc" : "df_first") << "(ah, al, " << C(t.first) << ".h, " << C(t.first)
              << ".l, " << t.second << ");";
            started = true;
        }
        o << "\n      " << dst << " = df_norm(ah, al); }\n";
    };
    std::ostringstream o;
    o << "#define MLN_JIT 1\n"
      << "#ifdef __CUDACC_RTC__\ntypedef long long int64_t;\ntypedef int int32_t;\ntypedef unsigned int uint32_t;\n#endif\n"
      << kKernelsSource << "\nnamespace mln {\n"
      << "struct JitBatchConsts { Df c[" << ncp << "]; };\n"
      << "struct JitBatchCell {\n  static constexpr int D = " << D << ";\n  using Consts = JitBatchConsts;\n"
      << "  using Field = Df;\n  Df s[D];\n";
    if (regs) o << "  Df c[" << nc << "];\n";
    o << "  __device__ __forceinline__ void setup(unsigned char *, const Consts &k) {";
    if (regs) o << " for (int i = 0; i < " << nc << "; ++i) c[i] = k.c[i];";
    o << " }\n"
      << "  __device__ __forceinline__ void load(const double *src, int64_t stride, int64_t m) { for (int i = 0; i < D; "
         "++i) s[i] = df_of(src[i * stride + m]); }\n"
      << "  __device__ __forceinline__ void load_cg(const double *src, int64_t stride, int64_t m) { for (int i = 0; i < "
         "D; ++i) s[i] = df_of(__ldcg(src + i * stride + m)); }\n"
      << "  __device__ __forceinline__ void store(double *dst, int64_t stride, int64_t m) const { for (int i = 0; i < "
         "D; ++i) dst[i * stride + m] = df_value(s[i]); }\n"
      << "  __device__ __forceinline__ void end_step() {}\n"
      << "  __device__ __forceinline__ Df step(Df e, const Consts &k) {\n"
      << "    Df z[D], y[D];\n";
    for (int k = 0; k < P; ++k) {
        std::vector<std::pair<int, std::string>> t;
        for (int i = 0; i < D; ++i)
            if (pat.tt[k * D + i]) t.push_back({iT[i * P + k], "s[" + std::to_string(i) + "]"});
        row(o, "z[" + std::to_string(k) + "]", "", -1, t);
    }
    for (int k = P; k < D; ++k) o << "    z[" << k << "] = Df{0.0f, 0.0f};\n";
    o << "    const float psi_h[" << (N - 1) << "] = {";
    for (int a = 0; a < N - 1; ++a) o << (a ? ", " : "") << C(iPsi[a]) << ".h";
    o << "}, psi_l[" << (N - 1) << "] = {";
    for (int a = 0; a < N - 1; ++a) o << (a ? ", " : "") << C(iPsi[a]) << ".l";
    o << "};\n    df_rotation_increment<" << N << ">(z, psi_h, psi_l, e);\n";
    for (int i = 0; i < D; ++i) {
        std::vector<std::pair<int, std::string>> t;
        for (int p = 0; p < P; ++p)
            if (pat.t[i * P + p]) t.push_back({iT[i * P + p], "z[" + std::to_string(p) + "]"});
        row(o, "y[" + std::to_string(i) + "]", "s[" + std::to_string(i) + "]", -1, t);
    }
    {
        std::vector<std::pair<int, std::string>> t;
        for (int i = 0; i < D; ++i)
            if (pat.wm[i]) t.push_back({iW[i], "y[" + std::to_string(i) + "]"});
        o << "    Df dpdt;\n";
        row(o, "dpdt", "", iCm, t);
    }
    for (int i = 0; i < D; ++i) {
        std::vector<std::pair<int, std::string>> t;
        for (int j = 0; j < D; ++j)
            if (pat.c1[i * D + j]) t.push_back({iC[i * D + j], "y[" + std::to_string(j) + "]"});
        row(o, "s[" + std::to_string(i) + "]", "y[" + std::to_string(i) + "]", iB[i], t);
    }
    const unsigned flags = pat.flags == ~0u ? 0u : pat.flags;
    o << "    return dpdt;\n  }\n};\n"
      << "extern \"C\" __global__ void __launch_bounds__(kBatchThreads, 1) mln_jit_batch(const BatchGrid<double> *grids, "
         "const BatchItem *items, const unsigned char *consts, int parity, int nsteps, int halo, int tile, "
         "int64_t step_offset) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  batch_body<" << N << ", double, JitBatchCell, " << flags
      << "u>(grids, items, consts, parity, nsteps, halo, tile, step_offset, smem_raw);\n}\n"
      << "extern \"C\" __global__ void __launch_bounds__(kBatchThreads, 1) mln_jit_batch_persist(const BatchGrid<double> "
         "*grids, const BatchItem *items, const unsigned char *consts, int halo, int tile, int64_t step_offset, "
         "BatchPersist p) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  batch_persistent<" << N << ", double, JitBatchCell, " << flags
      << "u>(grids, items, consts, halo, tile, step_offset, p, smem_raw);\n}\n"
      << "}  // namespace mln\n";
    return o.str();
}

bool jit_available(std::string *why) {
    std::lock_guard<std::mutex> lock(g_mu);
    bool ok = load_tools();
    if (!ok && why) *why = g_why;
    return ok;
}

cudaError_t jit_compile(const std::string &src, void **fn, std::string &log, const char *name) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!load_tools()) {
        log = g_why;
        return cudaErrorNotSupported;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_pair(dev, src);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {  // compiled before: look the kernel up by name
        CUfunction f = nullptr;
        if (g_drv.get(&f, it->second, name) != CUDA_SUCCESS) {
            log = std::string("no kernel ") + name + " in the compiled module";
            return cudaErrorUnknown;
        }
        *fn = f;
        return cudaSuccess;
    }
    nvrtcProgram_t prog = nullptr;
    if (g_nvrtc.create(&prog, src.c_str(), "mln_jit.cu", 0, nullptr, nullptr) != 0) {
        log = "nvrtcCreateProgram failed";
        return cudaErrorUnknown;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "-default-device"};
    int rc = g_nvrtc.compile(prog, 4, opts);
    size_t ls = 0;
    g_nvrtc.log_size(prog, &ls);
    std::string lg(ls, '\0');
    if (ls) g_nvrtc.log(prog, &lg[0]);
    if (rc != 0) {
        log = "NVRTC: " + lg;
        g_nvrtc.destroy(&prog);
        return cudaErrorUnknown;
    }
    size_t cs = 0;
    g_nvrtc.cubin_size(prog, &cs);
    std::vector<char> cubin(cs);
    g_nvrtc.cubin(prog, cubin.data());
    g_nvrtc.destroy(&prog);
    CUmodule mod = nullptr;
    CUfunction f = nullptr;
    if (g_drv.load(&mod, cubin.data()) != CUDA_SUCCESS || g_drv.get(&f, mod, name) != CUDA_SUCCESS) {
        log = "loading the compiled kernel failed";
        return cudaErrorUnknown;
    }
    g_cache[key] = mod;  // modules stay loaded until the process exits
    *fn = f;
    return cudaSuccess;
}

template <typename R>
cudaError_t jit_launch_t(void *fn, const BlockArgs<R> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st) {
    struct {
        int unused;
    } k{0};
    void *params[] = {const_cast<BlockArgs<R> *>(&a), &k};
    if (g_drv.launch_ex) {
        // programmatic dependency on the kernel before it in the stream: the
        // blocks are placed on SMs as the previous grid's blocks exit and start
        // as soon as that grid completes (the kernel waits for it first)
        CUlaunchAttribute attr[1];
        std::memset(attr, 0, sizeof(attr));
        attr[0].id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
        attr[0].value.programmaticStreamSerializationAllowed = 1;
        CUlaunchConfig cfg;
        std::memset(&cfg, 0, sizeof(cfg));
        cfg.gridDimX = g.x;
        cfg.gridDimY = g.y;
        cfg.gridDimZ = g.z;
        cfg.blockDimX = b.x;
        cfg.blockDimY = b.y;
        cfg.blockDimZ = b.z;
        cfg.sharedMemBytes = static_cast<unsigned>(smem);
        cfg.hStream = static_cast<CUstream>(st);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const CUresult r = g_drv.launch_ex(&cfg, static_cast<CUfunction>(fn), params, nullptr);
        return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
    }
    CUresult r = g_drv.launch(static_cast<CUfunction>(fn), g.x, g.y, g.z, b.x, b.y, b.z, static_cast<unsigned>(smem),
                              static_cast<CUstream>(st), params, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t jit_launch_batch(void *fn, const void *grids, const void *items, const void *consts, int parity,
                             int nsteps, int halo, int tile, int64_t step_offset, unsigned nblocks, unsigned threads,
                             size_t smem, cudaStream_t st) {
    void *params[] = {&grids, &items, &consts, &parity, &nsteps, &halo, &tile, &step_offset};
    CUresult r = g_drv.launch(static_cast<CUfunction>(fn), nblocks, 1, 1, threads, 1, 1, static_cast<unsigned>(smem),
                              static_cast<CUstream>(st), params, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t jit_launch_batch_persist(void *fn, const void *grids, const void *items, const void *consts, int halo,
                                     int tile, int64_t step_offset, const BatchPersist &p, unsigned nblocks,
                                     unsigned threads, size_t smem, cudaStream_t st) {
    BatchPersist pp = p;
    void *params[] = {&grids, &items, &consts, &halo, &tile, &step_offset, &pp};
    CUresult r = g_drv.launch(static_cast<CUfunction>(fn), nblocks, 1, 1, threads, 1, 1, static_cast<unsigned>(smem),
                              static_cast<CUstream>(st), params, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t jit_launch(void *fn, const BlockArgs<double> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st) {
    return jit_launch_t<double>(fn, a, g, b, smem, st);
}
cudaError_t jit_launch(void *fn, const BlockArgs<float> &a, dim3 g, dim3 b, size_t smem, cudaStream_t st) {
    return jit_launch_t<float>(fn, a, g, b, smem, st);
}

}  // namespace mln
