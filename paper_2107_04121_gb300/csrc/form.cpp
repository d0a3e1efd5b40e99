// Weak-form compiler: the generalized einsum-like notation of Tab. wfc of
// Cimrman, arXiv 2107.04121 (symbols 0, i, i.j, i:j, s(i:j)->I), one
// comma-separated subscript per operand, parsed into operand descriptors and
// matched against the forms that have GPU kernels (Tab. ewfd).  The result is
// kept in a handle, which plays the role of the cached transpilation result
// of Sec. 5.1 (Algorithm 3, "transpile").
#include <cctype>
#include <new>
#include <string>
#include <vector>

#include "fe_internal.h"

namespace {

enum SubKind { SK_SCALAR, SK_SCALAR_GRAD, SK_VEC, SK_VEC_GRAD, SK_SYMGRAD, SK_VOIGT, SK_MATERIAL };

struct Sub {
    SubKind kind;
    char a = 0, b = 0, c = 0;  // letters: component, derivative, storage
    std::string letters;       // material indices
};

bool is_letter(char ch) { return std::isalpha((unsigned char)ch) != 0; }

std::string strip(const std::string &s)
{
    size_t b = 0, e = s.size();
    while (b < e && std::isspace((unsigned char)s[b])) ++b;
    while (e > b && std::isspace((unsigned char)s[e - 1])) --e;
    return s.substr(b, e - b);
}

// Parse one field subscript; returns false on a syntax error.
bool parse_field(const std::string &t, Sub &out)
{
    const size_t n = t.size();
    if (t == "0") {
        out.kind = SK_SCALAR;
        return true;
    }
    if (n == 3 && t[0] == '0' && t[1] == '.' && is_letter(t[2])) {
        out.kind = SK_SCALAR_GRAD;
        out.b = t[2];
        return true;
    }
    if (n == 1 && is_letter(t[0])) {
        out.kind = SK_VEC;
        out.a = t[0];
        return true;
    }
    if (n == 3 && is_letter(t[0]) && (t[1] == '.' || t[1] == ':') && is_letter(t[2])) {
        out.kind = t[1] == '.' ? SK_VEC_GRAD : SK_SYMGRAD;
        out.a = t[0];
        out.b = t[2];
        return true;
    }
    // s(i:j)->I
    if (n == 9 && t[0] == 's' && t[1] == '(' && is_letter(t[2]) && t[3] == ':' && is_letter(t[4]) && t[5] == ')' &&
        t[6] == '-' && t[7] == '>' && is_letter(t[8])) {
        out.kind = SK_VOIGT;
        out.a = t[2];
        out.b = t[4];
        out.c = t[8];
        return true;
    }
    return false;
}

bool parse_material(const std::string &t, Sub &out)
{
    out.kind = SK_MATERIAL;
    if (t == "0") {
        out.letters.clear();
        return true;
    }
    if (t.empty() || t.size() > 4) return false;
    for (char ch : t)
        if (!is_letter(ch)) return false;
    out.letters = t;
    return true;
}

}  // namespace

extern "C" fe_status fe_form_compile(fe_ctx *ctx, const char *expr, const fe_operand *ops, int n_ops,
                                     fe_form_h **out)
{
    fe_clear_last_error();
    (void)ctx;
    if (!expr || !ops || !out || n_ops < 1 || n_ops > 8) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<std::string> parts;
    {
        std::string s(expr), cur;
        for (char ch : s) {
            if (ch == ',') {
                parts.push_back(strip(cur));
                cur.clear();
            } else {
                cur.push_back(ch);
            }
        }
        parts.push_back(strip(cur));
    }
    if ((int)parts.size() != n_ops) return FE_ERR_INVALID_ARG;

    std::vector<Sub> subs(n_ops);
    int iv = -1, im = -1;
    std::vector<int> states, params;
    for (int k = 0; k < n_ops; ++k) {
        const fe_operand &op = ops[k];
        if (op.role == FE_MATERIAL) {
            if (!parse_material(parts[k], subs[k])) return FE_ERR_INVALID_ARG;
            if (op.material != FE_MAT_SCALAR && op.material != FE_MAT_LAME && op.material != FE_MAT_D66 &&
                op.material != FE_MAT_M33)
                return FE_ERR_INVALID_ARG;
            if (im >= 0) return FE_ERR_UNSUPPORTED_SPEC;
            im = k;
        } else if (op.role == FE_VIRTUAL || op.role == FE_STATE || op.role == FE_PARAMETER) {
            if (!parse_field(parts[k], subs[k])) return FE_ERR_INVALID_ARG;
            if (op.ncomp != 1 && op.ncomp != 3) return FE_ERR_INVALID_ARG;
            if (op.material != FE_MAT_NONE) return FE_ERR_INVALID_ARG;
            // scalar symbols need a scalar field, component symbols a vector field
            const bool scalar_sym = subs[k].kind == SK_SCALAR || subs[k].kind == SK_SCALAR_GRAD;
            if (scalar_sym && op.ncomp != 1) return FE_ERR_INVALID_ARG;
            if (op.role == FE_VIRTUAL) {
                if (iv >= 0) return FE_ERR_UNSUPPORTED_SPEC;
                iv = k;
            } else if (op.role == FE_STATE) {
                states.push_back(k);
            } else {
                params.push_back(k);
            }
        } else {
            return FE_ERR_INVALID_ARG;
        }
    }
    // field operands in expression order; without a test function the form is
    // an 'eval' form and its first field takes the test function's place
    std::vector<int> fields;
    for (int k = 0; k < n_ops; ++k)
        if (ops[k].role != FE_MATERIAL) fields.push_back(k);
    if (fields.empty()) return FE_ERR_UNSUPPORTED_SPEC;
    const bool eval = iv < 0;
    const int ia = eval ? fields[0] : iv;
    std::vector<int> rest;
    for (int k : fields)
        if (k != ia) rest.push_back(k);

    fe_form_h f{};
    f.n_ops = n_ops;
    f.virtual_op = iv;
    f.state_op = states.empty() ? -1 : states[0];
    f.mat_op = im;
    f.mat = im >= 0 ? ops[im].material : FE_MAT_NONE;
    f.ncomp = ops[ia].ncomp;
    f.mat_transposed = 0;
    f.grad_op = f.adv_op = -1;
    f.eval = eval;
    f.op_a = ia;
    f.op_b = rest.empty() ? -1 : rest[0];
    f.op_c = rest.size() > 1 ? rest[1] : -1;
    f.ncomp_test = ops[ia].ncomp;
    f.ncomp_trial = rest.empty() ? 0 : ops[rest[0]].ncomp;
    f.n_out = 1;
    const Sub &V = subs[ia];
    bool ok = false;

    auto finish = [&]() -> fe_status {
        fe_form_h *h = new (std::nothrow) fe_form_h(f);
        if (!h) return FE_ERR_OOM;
        *out = h;
        return FE_OK;
    };

    // Navier-Stokes convection v_i (du_i/dx_j) w_j: a vector test slot, one
    // gradient operand with its component letter and one advection operand
    // carrying the derivative letter; u and w are each FE_STATE or FE_PARAMETER
    if (im < 0 && rest.size() == 2 && V.kind == SK_VEC && ops[ia].ncomp == 3) {
        int og = -1, oa = -1;
        for (int k : rest) {
            if (subs[k].kind == SK_VEC_GRAD) og = k;
            else if (subs[k].kind == SK_VEC) oa = k;
        }
        if (og >= 0 && oa >= 0 && ops[og].ncomp == 3 && ops[oa].ncomp == 3) {
            const Sub &Gs = subs[og], &A = subs[oa];
            if (Gs.a == V.a && A.a == Gs.b && Gs.a != Gs.b) {
                f.kind = FK_CONVECT;
                f.grad_op = og;
                f.adv_op = oa;
                f.wrt_grad = ops[og].role == FE_STATE;
                f.wrt_adv = ops[oa].role == FE_STATE;
                f.state_op = states.empty() ? -1 : states[0];
                f.ncomp_trial = 3;
                if (!eval && states.empty()) return FE_ERR_UNSUPPORTED_SPEC;
                return finish();
            }
        }
        return FE_ERR_UNSUPPORTED_SPEC;
    }
    // divergence div(v): a single vector field with the trace symbol
    if (im < 0 && rest.empty()) {
        if (V.kind == SK_VEC_GRAD && V.a == V.b && ops[ia].ncomp == 3) {
            f.kind = FK_DIV;
            return finish();
        }
        return FE_ERR_UNSUPPORTED_SPEC;
    }
    // Cauchy stress D_IK e_K(u): evaluated only (it has no test function)
    if (im >= 0 && rest.empty()) {
        const std::string &L = subs[im].letters;
        if (eval && V.kind == SK_VOIGT && ops[ia].ncomp == 3 && L.size() == 2 && L[0] != L[1] &&
            (ops[im].material == FE_MAT_LAME || ops[im].material == FE_MAT_D66) && V.a != V.b && V.a != V.c &&
            V.b != V.c && (L[1] == V.c || L[0] == V.c)) {
            f.kind = FK_CAUCHY;
            f.mat_transposed = L[0] == V.c;
            f.n_out = 6;
            return finish();
        }
        return FE_ERR_UNSUPPORTED_SPEC;
    }
    if (rest.size() != 1) return FE_ERR_UNSUPPORTED_SPEC;
    // bilinear forms: the weak forms need one unknown and no known field
    const int ib = rest[0];
    if (!eval && (states.size() != 1 || !params.empty() || states[0] != ib)) return FE_ERR_UNSUPPORTED_SPEC;
    const Sub &S = subs[ib];
    const int nc = ops[ia].ncomp;
    const bool scalar_mat = im < 0 || (subs[im].letters.empty() && ops[im].material == FE_MAT_SCALAR);

    // weak Laplacian: grad v . grad u, with an optional scalar coefficient
    if (V.kind == SK_SCALAR_GRAD && S.kind == SK_SCALAR_GRAD && V.b == S.b && scalar_mat) {
        f.kind = FK_LAPLACE;
        ok = true;
    }
    // dot product / mass: v_i u_i or scalar v u, optional scalar coefficient
    if (!ok && scalar_mat && ops[ib].ncomp == nc &&
        ((V.kind == SK_SCALAR && S.kind == SK_SCALAR) || (V.kind == SK_VEC && S.kind == SK_VEC && V.a == S.a))) {
        f.kind = FK_MASS;
        ok = true;
    }
    // weighted dot product v_i M_ij u_j
    if (!ok && im >= 0 && ops[im].material == FE_MAT_M33 && V.kind == SK_VEC && S.kind == SK_VEC && V.a != S.a &&
        nc == 3 && ops[ib].ncomp == 3) {
        const std::string &L = subs[im].letters;
        if (L.size() == 2 && L[0] == V.a && L[1] == S.a) {
            f.kind = FK_WDOT;
            ok = true;
        } else if (L.size() == 2 && L[0] == S.a && L[1] == V.a) {
            f.kind = FK_WDOT;
            f.mat_transposed = 1;
            ok = true;
        }
    }
    // Stokes coupling div(v) p and its transpose q div(u)
    if (!ok && im < 0 && V.kind == SK_VEC_GRAD && V.a == V.b && nc == 3 && S.kind == SK_SCALAR &&
        ops[ib].ncomp == 1) {
        f.kind = FK_STOKES;
        ok = true;
    }
    if (!ok && im < 0 && V.kind == SK_SCALAR && nc == 1 && S.kind == SK_VEC_GRAD && S.a == S.b &&
        ops[ib].ncomp == 3) {
        f.kind = FK_STOKES_T;
        ok = true;
    }
    // linear elasticity: D_IK e_I(v) e_K(u) in Voigt storage
    if (!ok && im >= 0 && V.kind == SK_VOIGT && S.kind == SK_VOIGT && nc == 3 && ops[ib].ncomp == 3 &&
        (ops[im].material == FE_MAT_LAME || ops[im].material == FE_MAT_D66) && subs[im].letters.size() == 2) {
        const std::string &L = subs[im].letters;
        // the symmetric-gradient letters are bound inside s(...): all four distinct,
        // and different from the storage letters
        const std::string inner{V.a, V.b, S.a, S.b};
        bool distinct = V.c != S.c && L[0] != L[1];
        for (int x = 0; x < 4 && distinct; ++x)
            for (int y = x + 1; y < 4; ++y)
                if (inner[x] == inner[y]) distinct = false;
        for (char ch : inner)
            if (ch == V.c || ch == S.c) distinct = false;
        if (distinct && L[0] == V.c && L[1] == S.c) {
            f.kind = FK_ELASTICITY;
            ok = true;
        } else if (distinct && L[0] == S.c && L[1] == V.c) {
            f.kind = FK_ELASTICITY;
            f.mat_transposed = 1;
            ok = true;
        }
    }
    if (!ok) return FE_ERR_UNSUPPORTED_SPEC;
    return finish();
}

extern "C" fe_status fe_form_free(fe_form_h *form)
{
    fe_clear_last_error();
    delete form;
    return FE_OK;
}

extern "C" fe_status fe_form_shape(const fe_form_h *form, int n_basis, int *n_rows, int *n_cols)
{
    fe_clear_last_error();
    if (!form || n_basis < 1) return FE_ERR_INVALID_ARG;
    if (form->eval) {
        if (n_rows) *n_rows = form->n_out;
        if (n_cols) *n_cols = 0;
        return FE_OK;
    }
    if (n_rows) *n_rows = form->ncomp_test * n_basis;
    if (n_cols) *n_cols = form->kind == FK_DIV ? 0 : form->ncomp_trial * n_basis;
    return FE_OK;
}
