// qasm.cpp — OpenQASM 2.0 front-end (the circuit input of Sec. 4.1: a QASM file is
// read into a flat gate list, from which Step A builds the dependency graph).
//
// Subset: the header and include lines, qreg / creg declarations (several quantum
// registers are laid out one after another), gate calls on single qubits or on whole
// registers (applied element-wise), parameter expressions (numbers, pi, + - * / ^,
// unary minus, parentheses, sin cos tan exp ln sqrt), and the qelib1 gates this
// library executes: id u u1 u2 u3 U p x y z h s sdg t tdg rx ry rz cx CX cy cz cp cu1
// swap rzz (rzz(t) a,b is emitted as CX(a,b) RZ(t)(b) CX(a,b), the same unitary).
// measure and barrier are accepted and emit nothing (measurement is not simulated).
// Gate definitions, opaque gates, reset and classically controlled gates are rejected
// with a message naming the line.
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "planner.h"
#include "sv.h"

namespace {

struct Tok {
    enum Kind { END, ID, NUM, STR, SYM } k = END;
    std::string s;
    double v = 0;
    int line = 1;
};

class Lexer {
  public:
    explicit Lexer(const char* p) : p_(p) {}
    Tok next() {
        skip();
        Tok t;
        t.line = line_;
        if (!*p_) return t;
        const char c = *p_;
        if (std::isalpha((unsigned char)c) || c == '_') {
            const char* b = p_;
            while (std::isalnum((unsigned char)*p_) || *p_ == '_') ++p_;
            t.k = Tok::ID;
            t.s.assign(b, p_);
        } else if (std::isdigit((unsigned char)c) || (c == '.' && std::isdigit((unsigned char)p_[1]))) {
            char* e = nullptr;
            t.v = std::strtod(p_, &e);
            t.k = Tok::NUM;
            t.s.assign(p_, static_cast<const char*>(e));
            p_ = e;
        } else if (c == '"') {
            const char* b = ++p_;
            while (*p_ && *p_ != '"') ++p_;
            t.k = Tok::STR;
            t.s.assign(b, p_);
            if (*p_) ++p_;
        } else if (c == '-' && p_[1] == '>') {
            t.k = Tok::SYM;
            t.s = "->";
            p_ += 2;
        } else if (c == '=' && p_[1] == '=') {
            t.k = Tok::SYM;
            t.s = "==";
            p_ += 2;
        } else {
            t.k = Tok::SYM;
            t.s = std::string(1, c);
            ++p_;
        }
        return t;
    }

  private:
    const char* p_;
    int line_ = 1;
    void skip() {
        for (;;) {
            while (*p_ && std::isspace((unsigned char)*p_)) {
                if (*p_ == '\n') ++line_;
                ++p_;
            }
            if (p_[0] == '/' && p_[1] == '/') {
                while (*p_ && *p_ != '\n') ++p_;
                continue;
            }
            if (p_[0] == '/' && p_[1] == '*') {
                p_ += 2;
                while (*p_ && !(p_[0] == '*' && p_[1] == '/')) {
                    if (*p_ == '\n') ++line_;
                    ++p_;
                }
                if (*p_) p_ += 2;
                continue;
            }
            break;
        }
    }
};

struct Arg {
    int reg;     // register index
    int idx;     // -1: whole register
};

class Parser {
  public:
    explicit Parser(const char* text) : lx_(text) { adv(); }
    std::string run(std::vector<sv_gate>* out, uint32_t* nq);

  private:
    Lexer lx_;
    Tok t_;
    std::vector<std::pair<std::string, int>> qregs_;   // name, size (in order)
    std::map<std::string, int> creg_;
    std::vector<sv_gate>* out_ = nullptr;

    void adv() { t_ = lx_.next(); }
    bool sym(const char* s) const { return t_.k == Tok::SYM && t_.s == s; }
    std::string where() const { return "line " + std::to_string(t_.line) + ": "; }
    std::string expect(const char* s) {
        if (!sym(s)) return where() + "expected '" + s + "'";
        adv();
        return "";
    }
    int qreg(const std::string& name) const {
        for (size_t i = 0; i < qregs_.size(); ++i)
            if (qregs_[i].first == name) return (int)i;
        return -1;
    }
    int offset(int reg) const {
        int o = 0;
        for (int i = 0; i < reg; ++i) o += qregs_[i].second;
        return o;
    }
    // expressions (OpenQASM 2: +, -, *, /, ^, unary -, functions, pi)
    std::string expr(double* v);
    std::string term(double* v);
    std::string factor(double* v);
    std::string atom(double* v);
    std::string args(std::vector<Arg>* a, bool quantum);
    std::string emit(const std::string& name, const std::vector<double>& p, const std::vector<Arg>& a);
    void put(int kind, int q0, int q1, double a0 = 0, double a1 = 0, double a2 = 0) {
        sv_gate g;
        std::memset(&g, 0, sizeof(g));
        g.kind = (uint16_t)kind;
        g.nq = (uint8_t)(q1 < 0 ? 1 : 2);
        g.q[0] = (uint8_t)q0;
        g.q[1] = (uint8_t)(q1 < 0 ? 0 : q1);
        g.param = -1;
        g.angle[0] = a0;
        g.angle[1] = a1;
        g.angle[2] = a2;
        out_->push_back(g);
    }
};

std::string Parser::atom(double* v) {
    if (t_.k == Tok::NUM) {
        *v = t_.v;
        adv();
        return "";
    }
    if (t_.k == Tok::ID) {
        const std::string id = t_.s;
        adv();
        if (id == "pi") {
            *v = M_PI;
            return "";
        }
        static const char* fns[] = {"sin", "cos", "tan", "exp", "ln", "sqrt"};
        for (const char* f : fns)
            if (id == f) {
                std::string e = expect("(");
                if (e.empty()) e = expr(v);
                if (e.empty()) e = expect(")");
                if (!e.empty()) return e;
                if (id == "sin") *v = std::sin(*v);
                else if (id == "cos") *v = std::cos(*v);
                else if (id == "tan") *v = std::tan(*v);
                else if (id == "exp") *v = std::exp(*v);
                else if (id == "ln") *v = std::log(*v);
                else *v = std::sqrt(*v);
                return "";
            }
        return where() + "unknown identifier '" + id + "' in an expression";
    }
    if (sym("(")) {
        adv();
        std::string e = expr(v);
        if (e.empty()) e = expect(")");
        return e;
    }
    return where() + "expected an expression";
}

std::string Parser::factor(double* v) {   // unary minus binds looser than ^
    if (sym("-")) {
        adv();
        std::string e = factor(v);
        *v = -*v;
        return e;
    }
    if (sym("+")) {
        adv();
        return factor(v);
    }
    std::string e = atom(v);
    if (!e.empty()) return e;
    if (sym("^")) {
        adv();
        double r = 0;
        e = factor(&r);
        if (!e.empty()) return e;
        *v = std::pow(*v, r);
    }
    return "";
}

std::string Parser::term(double* v) {
    std::string e = factor(v);
    while (e.empty() && (sym("*") || sym("/"))) {
        const bool mul = sym("*");
        adv();
        double r = 0;
        e = factor(&r);
        if (e.empty()) *v = mul ? *v * r : *v / r;
    }
    return e;
}

std::string Parser::expr(double* v) {
    std::string e = term(v);
    while (e.empty() && (sym("+") || sym("-"))) {
        const bool add = sym("+");
        adv();
        double r = 0;
        e = term(&r);
        if (e.empty()) *v = add ? *v + r : *v - r;
    }
    return e;
}

std::string Parser::args(std::vector<Arg>* a, bool quantum) {
    for (;;) {
        if (t_.k != Tok::ID) return where() + "expected a register name";
        const std::string name = t_.s;
        adv();
        Arg x{-1, -1};
        if (quantum) {
            x.reg = qreg(name);
            if (x.reg < 0) return where() + "unknown quantum register '" + name + "'";
        } else if (!creg_.count(name) && qreg(name) < 0) {
            return where() + "unknown register '" + name + "'";
        }
        if (sym("[")) {
            adv();
            if (t_.k != Tok::NUM) return where() + "expected an index";
            x.idx = (int)t_.v;
            adv();
            std::string e = expect("]");
            if (!e.empty()) return e;
            if (quantum && (x.idx < 0 || x.idx >= qregs_[x.reg].second)) return where() + "index out of range";
        }
        a->push_back(x);
        if (!sym(",")) break;
        adv();
    }
    return "";
}

std::string Parser::emit(const std::string& name, const std::vector<double>& p, const std::vector<Arg>& a) {
    using namespace svh;
    struct G { const char* n; int kind; int nq; int np; };
    static const G table[] = {
        {"id", 0, 1, 0}, {"x", K_X, 1, 0}, {"y", K_Y, 1, 0}, {"z", K_Z, 1, 0}, {"h", K_H, 1, 0},
        {"s", K_S, 1, 0}, {"sdg", K_SDG, 1, 0}, {"t", K_T, 1, 0}, {"tdg", K_TDG, 1, 0},
        {"rx", K_RX, 1, 1}, {"ry", K_RY, 1, 1}, {"rz", K_RZ, 1, 1}, {"p", K_P, 1, 1}, {"u1", K_P, 1, 1},
        {"u2", K_U3, 1, 2}, {"u3", K_U3, 1, 3}, {"u", K_U3, 1, 3}, {"U", K_U3, 1, 3},
        {"cx", K_CX, 2, 0}, {"CX", K_CX, 2, 0}, {"cy", K_CY, 2, 0}, {"cz", K_CZ, 2, 0},
        {"cp", K_CP, 2, 1}, {"cu1", K_CP, 2, 1}, {"swap", K_SWAP, 2, 0}, {"rzz", -1, 2, 1},
    };
    const G* g = nullptr;
    for (const G& x : table)
        if (name == x.n) g = &x;
    if (!g) return where() + "unsupported gate '" + name + "'";
    if ((int)p.size() != g->np) return where() + "gate '" + name + "' takes " + std::to_string(g->np) + " parameters";
    if ((int)a.size() != g->nq) return where() + "gate '" + name + "' takes " + std::to_string(g->nq) + " qubits";
    // element-wise application over whole-register arguments
    int width = 1;
    for (const Arg& x : a)
        if (x.idx < 0) {
            const int sz = qregs_[x.reg].second;
            if (width != 1 && sz != width) return where() + "register sizes differ";
            width = sz;
        }
    for (int i = 0; i < width; ++i) {
        int q[2] = {-1, -1};
        for (int k = 0; k < g->nq; ++k) q[k] = offset(a[k].reg) + (a[k].idx < 0 ? i : a[k].idx);
        if (g->nq == 2 && q[0] == q[1]) return where() + "two-qubit gate on one qubit";
        if (g->kind == 0) continue;   // identity
        if (g->kind < 0) {            // rzz(t) = CX . (I x RZ(t)) . CX
            put(K_CX, q[0], q[1]);
            put(K_RZ, q[1], -1, p[0]);
            put(K_CX, q[0], q[1]);
        } else if (g->kind == K_U3 && g->np == 2) {   // u2(phi, lambda) = u3(pi/2, phi, lambda)
            put(K_U3, q[0], -1, M_PI / 2, p[0], p[1]);
        } else {
            put(g->kind, q[0], q[1], p.size() > 0 ? p[0] : 0.0, p.size() > 1 ? p[1] : 0.0, p.size() > 2 ? p[2] : 0.0);
        }
    }
    return "";
}

std::string Parser::run(std::vector<sv_gate>* out, uint32_t* nq) {
    out_ = out;
    while (t_.k != Tok::END) {
        if (t_.k != Tok::ID) return where() + "expected a statement";
        const std::string kw = t_.s;
        adv();
        std::string e;
        if (kw == "OPENQASM") {
            if (t_.k != Tok::NUM) return where() + "expected a version";
            adv();
            e = expect(";");
        } else if (kw == "include") {
            if (t_.k != Tok::STR) return where() + "expected a file name";
            adv();
            e = expect(";");
        } else if (kw == "qreg" || kw == "creg") {
            if (t_.k != Tok::ID) return where() + "expected a register name";
            const std::string name = t_.s;
            adv();
            if ((e = expect("[")).size()) return e;
            if (t_.k != Tok::NUM || t_.v < 1) return where() + "expected a register size";
            const int size = (int)t_.v;
            adv();
            if ((e = expect("]")).size()) return e;
            e = expect(";");
            if (kw == "qreg") {
                if (qreg(name) >= 0) return where() + "register '" + name + "' declared twice";
                qregs_.push_back({name, size});
            } else {
                creg_[name] = size;
            }
        } else if (kw == "barrier") {
            std::vector<Arg> a;
            if ((e = args(&a, true)).size()) return e;
            e = expect(";");
        } else if (kw == "measure") {
            std::vector<Arg> a, c;
            if ((e = args(&a, true)).size()) return e;
            if ((e = expect("->")).size()) return e;
            if ((e = args(&c, false)).size()) return e;
            e = expect(";");
        } else if (kw == "gate" || kw == "opaque" || kw == "reset" || kw == "if") {
            return where() + "'" + kw + "' is not supported (flat gate lists only)";
        } else {
            std::vector<double> p;
            if (sym("(")) {
                adv();
                if (!sym(")"))
                    for (;;) {
                        double v = 0;
                        if ((e = expr(&v)).size()) return e;
                        p.push_back(v);
                        if (!sym(",")) break;
                        adv();
                    }
                if ((e = expect(")")).size()) return e;
            }
            std::vector<Arg> a;
            if ((e = args(&a, true)).size()) return e;
            if ((e = emit(kw, p, a)).size()) return e;
            e = expect(";");
        }
        if (!e.empty()) return e;
    }
    int total = 0;
    for (auto& r : qregs_) total += r.second;
    if (total == 0) return "no quantum register declared";
    if (total > 255) return "more than 255 qubits";
    *nq = (uint32_t)total;
    return "";
}

}  // namespace

extern "C" sv_status sv_qasm_parse(const char* text, sv_gate* gates, uint32_t capacity, uint32_t* n_qubits,
                                   uint32_t* n_gates) {
    if (!text || !n_qubits || !n_gates) return svh::set_error(SV_ERR_ARG, "null argument");
    std::vector<sv_gate> out;
    uint32_t nq = 0;
    Parser P(text);
    std::string err = P.run(&out, &nq);
    if (!err.empty()) return svh::set_error(SV_ERR_ARG, err.c_str());
    *n_qubits = nq;
    *n_gates = (uint32_t)out.size();
    if (gates) {
        if (capacity < out.size()) return svh::set_error(SV_ERR_ARG, "gate array too small");
        std::memcpy(gates, out.data(), out.size() * sizeof(sv_gate));
    }
    return SV_OK;
}
