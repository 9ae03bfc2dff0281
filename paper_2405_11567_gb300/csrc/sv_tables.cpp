// sv_tables.cpp -- host construction of the excitation descriptors and of the
// Hamiltonian's X-mask tables.
//
// The Hamiltonian (FCIDUMP chemist notation, Methodology "Computational
// Details") is grouped by flip mask m = x ^ x': after the Jordan-Wigner mapping
// every Pauli string with X-part m connects x to x ^ m, and the sum of all the
// strings that share m, evaluated at x, is the matrix element <x^m|H|x>.  Here that
// sum is evaluated in closed form (Slater-Condon rules) rather than string by
// string:
//   m = 0 (diagonal):   E_nuc + sum_k x_k h_kk + sum_{k<l} x_k x_l ([kk|ll] - [kl|lk])
//   m = {i, a} (single, same spin), x with one of the two bits set:
//                       (-1)^popc(x & between(i,a)) (h_ai + sum_{k != i,a} x_k ([ai|kk] - [ak|ki]))
//   m = {q0<q1<q2<q3} (double), x with two of the four bits set, occupied i<j,
//                       empty a<b:   (-1)^popc(x & sm) ([ai|bj] - [aj|bi])
//                       sm = between(q0,q1) | between(q2,q3)
// with [PQ|RS] = (pq|rs) delta(spin P, spin Q) delta(spin R, spin S).  The sign
// masks follow from applying a+_a a+_b a_j a_i literally with the Jordan-Wigner
// string on lower indices: the parity of the occupied orbitals strictly between
// i and j plus those strictly between a and b, with i and j themselves excluded,
// which for every way of splitting {q0..q3} into an occupied and an empty pair is
// the parity on between(q0,q1) | between(q2,q3).
#include <algorithm>
#include <cmath>
#include <string>

#include "sv_internal.h"

namespace svk {

static bool make_op_qubits(const sv_excitation &e, int n, OpDesc &d, std::string &why) {
    auto inrange = [&](int v) { return v >= 0 && v < n; };
    d = OpDesc();
    if (e.kind == 1 || e.kind == 3) {
        int i = e.occ[0], a = e.vir[0];
        if (!inrange(i) || !inrange(a)) { why = "single excitation index out of range"; return false; }
        if (i == a) { why = "single excitation with occ == vir"; return false; }
        if ((i & 1) != (a & 1)) { why = "single excitation does not conserve S_z"; return false; }
        d.nbits = 2;
        d.m = (1u << i) | (1u << a);
        d.from = 1u << i;  // T = a+_a a_i acts on x with i occupied, a empty
        d.sm = e.kind == 1 ? bits_between(i, a) : 0u;  // qubit excitation: no string, sign +1
        d.pos[0] = std::min(i, a);
        d.pos[1] = std::max(i, a);
        return true;
    }
    if (e.kind == 2 || e.kind == 4) {
        int i = e.occ[0], j = e.occ[1], a = e.vir[0], b = e.vir[1];
        if (!inrange(i) || !inrange(j) || !inrange(a) || !inrange(b)) {
            why = "double excitation index out of range"; return false;
        }
        if (!(i < j) || !(a < b)) { why = "double excitation needs occ[0] < occ[1] and vir[0] < vir[1]"; return false; }
        if (i == a || i == b || j == a || j == b) { why = "double excitation indices must be distinct"; return false; }
        int na_occ = ((i & 1) == 0) + ((j & 1) == 0), na_vir = ((a & 1) == 0) + ((b & 1) == 0);
        if (na_occ != na_vir) { why = "double excitation does not conserve S_z"; return false; }
        d.nbits = 4;
        d.m = (1u << i) | (1u << j) | (1u << a) | (1u << b);
        d.from = (1u << i) | (1u << j);
        int q[4] = {i, j, a, b};
        std::sort(q, q + 4);
        for (int t = 0; t < 4; ++t) d.pos[t] = q[t];
        d.sm = e.kind == 2 ? (bits_between(q[0], q[1]) | bits_between(q[2], q[3])) : 0u;
        return true;
    }
    why = "excitation kind must be 1, 2 (fermionic) or 3, 4 (qubit)";
    return false;
}

bool make_op(const sv_excitation &e, int n, const int *perm, OpDesc &d, std::string &why) {
    if (!make_op_qubits(e, n, d, why)) return false;
    // the sign is a parity of popcounts, invariant under relabelling the bits
    int pos[4];
    for (int t = 0; t < d.nbits; ++t) pos[t] = perm[d.pos[t]];
    std::sort(pos, pos + d.nbits);
    for (int t = 0; t < d.nbits; ++t) d.pos[t] = pos[t];
    d.m = map_bits(d.m, perm);
    d.from = map_bits(d.from, perm);
    d.sm = map_bits(d.sm, perm);
    return true;
}

template <typename R>
void permute_tables(HostTables<R> &t, const int *perm, int n) {
    for (auto &r : t.dbl) {
        r.m = map_bits(r.m, perm);
        r.sm = map_bits(r.sm, perm);
        r.b0 = map_bits(r.b0, perm);
        r.b1 = map_bits(r.b1, perm);
        r.b2 = map_bits(r.b2, perm);
    }
    for (auto &r : t.sgl) {
        r.m = map_bits(r.m, perm);
        r.sm = map_bits(r.sm, perm);
    }
    std::vector<R> W(t.W.size());
    for (size_t i = 0; i < t.sgl.size(); ++i)
        for (int k = 0; k < n; ++k) W[i * n + perm[k]] = t.W[i * n + k];
    t.W.swap(W);
    t.hdiag_s.assign(n, 0.0);
    t.Jp_s.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        t.hdiag_s[perm[k]] = t.hdiag[k];
        for (int l = 0; l < n; ++l) t.Jp_s[(size_t)perm[k] * n + perm[l]] = t.Jp[(size_t)k * n + l];
    }
}

template void permute_tables<float>(HostTables<float> &, const int *, int);
template void permute_tables<double>(HostTables<double> &, const int *, int);

template <typename R>
void build_tables(const sv_ham &H, int n, HostTables<R> &out) {
    const int N = H.n_orb;
    auto g = [&](int P, int Q, int Rr, int S) -> double {
        if ((P & 1) != (Q & 1) || (Rr & 1) != (S & 1)) return 0.0;
        size_t e = (((size_t)(P >> 1) * N + (Q >> 1)) * N + (Rr >> 1)) * N + (S >> 1);
        return H.eri[e];
    };
    auto hh = [&](int P, int Q) -> double {
        if ((P & 1) != (Q & 1)) return 0.0;
        return H.h[(size_t)(P >> 1) * N + (Q >> 1)];
    };
    out.dbl.clear();
    out.sgl.clear();
    out.W.clear();
    out.hdiag.assign(n, 0.0);
    out.Jp.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        out.hdiag[k] = hh(k, k);
        for (int l = 0; l < n; ++l)
            if (k != l) out.Jp[(size_t)k * n + l] = g(k, k, l, l) - g(k, l, l, k);
    }
    // singles: i < a, same spin
    for (int i = 0; i < n; ++i) {
        for (int a = i + 1; a < n; ++a) {
            if ((i & 1) != (a & 1)) continue;
            SingleRec<R> r;
            r.m = (1u << i) | (1u << a);
            r.sm = bits_between(i, a);
            r.h = (R)hh(a, i);
            r.pad = (R)0;
            bool any = r.h != (R)0;
            std::vector<R> w(n, (R)0);
            for (int k = 0; k < n; ++k) {
                if (k == i || k == a) continue;
                w[k] = (R)(g(a, i, k, k) - g(a, k, k, i));
                if (w[k] != (R)0) any = true;
            }
            if (!any) continue;
            out.sgl.push_back(r);
            out.W.insert(out.W.end(), w.begin(), w.end());
        }
    }
    // doubles: q0 < q1 < q2 < q3 with an even number of alpha spin-orbitals
    for (int q0 = 0; q0 < n; ++q0)
        for (int q1 = q0 + 1; q1 < n; ++q1)
            for (int q2 = q1 + 1; q2 < n; ++q2)
                for (int q3 = q2 + 1; q3 < n; ++q3) {
                    int nalpha = ((q0 & 1) == 0) + ((q1 & 1) == 0) + ((q2 & 1) == 0) + ((q3 & 1) == 0);
                    if (nalpha & 1) continue;
                    // split s: occupied pair contains q0 and q_{s+1}
                    const int occ[3][2] = {{q0, q1}, {q0, q2}, {q0, q3}};
                    const int emp[3][2] = {{q2, q3}, {q1, q3}, {q1, q2}};
                    DoubleRec<R> r;
                    r.m = (1u << q0) | (1u << q1) | (1u << q2) | (1u << q3);
                    r.sm = bits_between(q0, q1) | bits_between(q2, q3);
                    r.b0 = 1u << q0;
                    r.b1 = 1u << q1;
                    r.b2 = 1u << q2;
                    r.pad = 0;
                    bool any = false;
                    for (int s = 0; s < 3; ++s) {
                        int i = occ[s][0], j = occ[s][1], a = emp[s][0], b = emp[s][1];
                        double v = g(a, i, b, j) - g(a, j, b, i);
                        r.v[s] = (R)v;
                        if (r.v[s] != (R)0) any = true;
                    }
                    if (any) out.dbl.push_back(r);
                }
}

template void build_tables<float>(const sv_ham &, int, HostTables<float> &);
template void build_tables<double>(const sv_ham &, int, HostTables<double> &);

// Diagonal element <x|H|x> in float64 (used on the host for the shift constant).
double diag_energy(const sv_ham &H, uint32_t x, int n) {
    const int N = H.n_orb;
    double e = H.e_nuc;
    for (int k = 0; k < n; ++k) {
        if (!((x >> k) & 1)) continue;
        e += H.h[(size_t)(k >> 1) * N + (k >> 1)];
        for (int l = k + 1; l < n; ++l) {
            if (!((x >> l) & 1)) continue;
            size_t kkll = (((size_t)(k >> 1) * N + (k >> 1)) * N + (l >> 1)) * N + (l >> 1);
            e += H.eri[kkll];
            if ((k & 1) == (l & 1)) {
                size_t kllk = (((size_t)(k >> 1) * N + (l >> 1)) * N + (l >> 1)) * N + (k >> 1);
                e -= H.eri[kllk];
            }
        }
    }
    return e;
}

}  // namespace svk
