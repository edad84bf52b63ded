// Grammar compiler of the CUDA library: WCNF text -> production tables.
// Paper Sec. 2 (WCNF definition), appendix B (indexed non-terminals and the
// hand-made WCNF grammars of optimisation 5).
#include "grammar.h"

#include <algorithm>
#include <map>
#include <set>
#include <sstream>
#include <tuple>
#include <unordered_map>

namespace cflr {

int Grammar::find_nt(const std::string &s) const {
    for (size_t i = 0; i < nts.size(); i++)
        if (nts[i] == s) return (int)i;
    return -1;
}

int Grammar::find_term(const std::string &s) const {
    for (size_t i = 0; i < terms.size(); i++)
        if (terms[i] == s) return (int)i;
    return -1;
}

namespace {

struct RawProd {
    int line;
    std::vector<std::string> toks;   // toks[0] = lhs
    int32_t fam = -1;                // family of an expanded copy (see Grammar)
    uint32_t member = 0;
};

std::vector<std::string> split_ws(const std::string &s) {
    std::vector<std::string> out;
    std::istringstream is(s);
    std::string t;
    while (is >> t) out.push_back(t);
    return out;
}

// Index variables "_{v}" mentioned in a token.
void index_vars(const std::string &t, std::set<std::string> &vars) {
    size_t p = 0;
    while ((p = t.find("_{", p)) != std::string::npos) {
        size_t q = t.find('}', p + 2);
        if (q == std::string::npos) break;
        vars.insert(t.substr(p + 2, q - p - 2));
        p = q + 1;
    }
}

std::string substitute(const std::string &t, const std::map<std::string, long> &val) {
    std::string out;
    size_t p = 0;
    while (p < t.size()) {
        size_t s = t.find("_{", p);
        if (s == std::string::npos) { out += t.substr(p); break; }
        size_t q = t.find('}', s + 2);
        if (q == std::string::npos) { out += t.substr(p); break; }
        out += t.substr(p, s - p);
        auto it = val.find(t.substr(s + 2, q - s - 2));
        out += "_" + std::to_string(it->second);
        p = q + 1;
    }
    return out;
}

}  // namespace

int parse_grammar(const char *text, size_t len, Grammar &g, std::string &err) {
    g = Grammar();
    std::string src(text, len);
    std::istringstream lines(src);
    std::string line;
    int ln = 0;
    std::map<std::string, std::pair<long, long>> ranges;
    std::vector<RawProd> raw;
    while (std::getline(lines, line)) {
        ln++;
        size_t hash = line.find('#');
        if (hash != std::string::npos) line = line.substr(0, hash);
        std::vector<std::string> w = split_ws(line);
        if (w.empty()) continue;
        if (w[0][0] == '%') {
            if (w[0] != "%index" || w.size() != 4) {
                err = "line " + std::to_string(ln) + ": unknown or malformed directive";
                return -1;
            }
            char *e1 = nullptr, *e2 = nullptr;
            long lo = std::strtol(w[2].c_str(), &e1, 10), hi = std::strtol(w[3].c_str(), &e2, 10);
            if (*e1 || *e2 || hi < lo || hi - lo > 1000000) {
                err = "line " + std::to_string(ln) + ": bad %index range";
                return -1;
            }
            ranges[w[1]] = {lo, hi};
            continue;
        }
        size_t arrow = line.find("->");
        if (arrow == std::string::npos) {
            err = "line " + std::to_string(ln) + ": expected 'LHS -> ...'";
            return -1;
        }
        std::vector<std::string> lhs = split_ws(line.substr(0, arrow));
        if (lhs.size() != 1) {
            err = "line " + std::to_string(ln) + ": the left-hand side must be one symbol";
            return -1;
        }
        std::string rhs = line.substr(arrow + 2);
        size_t start = 0;
        for (;;) {
            size_t bar = rhs.find('|', start);
            std::string alt = rhs.substr(start, bar == std::string::npos ? std::string::npos
                                                                         : bar - start);
            std::vector<std::string> syms = split_ws(alt);
            if (syms.empty()) {
                err = "line " + std::to_string(ln) + ": empty alternative (write eps)";
                return -1;
            }
            RawProd rp;
            rp.line = ln;
            rp.toks.push_back(lhs[0]);
            rp.toks.insert(rp.toks.end(), syms.begin(), syms.end());
            raw.push_back(rp);
            if (bar == std::string::npos) break;
            start = bar + 1;
        }
    }

    // Expand indexed productions: one copy per assignment of their variables.
    // The copies of a line with one variable form a family.
    std::vector<RawProd> prods;
    std::vector<uint32_t> fam_size;
    for (const RawProd &rp : raw) {
        std::set<std::string> vars;
        for (const auto &t : rp.toks) index_vars(t, vars);
        std::vector<std::string> vs(vars.begin(), vars.end());
        for (const auto &v : vs)
            if (!ranges.count(v)) {
                err = "line " + std::to_string(rp.line) + ": index variable '" + v +
                      "' has no %index directive";
                return -1;
            }
        std::map<std::string, long> cur;
        for (const auto &v : vs) cur[v] = ranges[v].first;
        int32_t fam = -1;
        if (vs.size() == 1 && ranges[vs[0]].second > ranges[vs[0]].first) {
            fam = (int32_t)fam_size.size();
            fam_size.push_back((uint32_t)(ranges[vs[0]].second - ranges[vs[0]].first + 1));
        }
        for (;;) {
            RawProd e;
            e.line = rp.line;
            for (const auto &t : rp.toks) e.toks.push_back(substitute(t, cur));
            if (fam >= 0) {
                e.fam = fam;
                e.member = (uint32_t)(cur[vs[0]] - ranges[vs[0]].first);
            }
            prods.push_back(e);
            // odometer increment over the variables
            size_t k = 0;
            for (; k < vs.size(); k++) {
                if (++cur[vs[k]] <= ranges[vs[k]].second) break;
                cur[vs[k]] = ranges[vs[k]].first;
            }
            if (k == vs.size()) break;
        }
    }

    // Non-terminals: every left-hand side, in order of first appearance.
    std::unordered_map<std::string, uint32_t> nt_id;
    for (const RawProd &p : prods) {
        if (p.toks[0] == "eps") {
            err = "line " + std::to_string(p.line) + ": eps cannot be a left-hand side";
            return -1;
        }
        if (!nt_id.count(p.toks[0])) {
            nt_id[p.toks[0]] = (uint32_t)g.nts.size();
            g.nts.push_back(p.toks[0]);
        }
    }
    g.n_named = (uint32_t)g.nts.size();
    std::unordered_map<std::string, uint32_t> term_id;
    auto term_of = [&](const std::string &s) {
        auto it = term_id.find(s);
        if (it != term_id.end()) return it->second;
        uint32_t id = (uint32_t)g.terms.size();
        term_id[s] = id;
        g.terms.push_back(s);
        g.term_nts.emplace_back();
        return id;
    };
    std::unordered_map<std::string, uint32_t> wrapper;
    auto operand = [&](const std::string &s) -> uint32_t {
        auto it = nt_id.find(s);
        if (it != nt_id.end()) return it->second;
        auto w = wrapper.find(s);
        if (w != wrapper.end()) return w->second;
        uint32_t id = (uint32_t)g.nts.size();
        g.nts.push_back("<" + s + ">");
        wrapper[s] = id;
        g.term_nts[term_of(s)].push_back(id);   // "<x> -> x"
        return id;
    };

    std::set<std::tuple<uint32_t, uint32_t, uint32_t>> bin;
    // (c, a, b) -> (family, member); a production that two lines yield keeps
    // no family (-2 marks the clash)
    std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::pair<int32_t, uint32_t>> famof;
    std::set<std::pair<uint32_t, uint32_t>> unit;
    std::set<uint32_t> eps;
    for (const RawProd &p : prods) {
        uint32_t c = nt_id[p.toks[0]];
        size_t r = p.toks.size() - 1;
        if (r == 1 && p.toks[1] == "eps") {
            eps.insert(c);
        } else if (r == 1) {
            auto it = nt_id.find(p.toks[1]);
            if (it != nt_id.end()) unit.insert({c, it->second});
            else g.term_nts[term_of(p.toks[1])].push_back(c);
        } else if (r == 2) {
            if (p.toks[1] == "eps" || p.toks[2] == "eps") {
                err = "line " + std::to_string(p.line) + ": eps inside a binary production";
                return -1;
            }
            uint32_t a = operand(p.toks[1]);
            uint32_t b = operand(p.toks[2]);
            const auto key = std::make_tuple(c, a, b);
            if (bin.insert(key).second) famof[key] = {p.fam, p.member};
            else famof[key] = {-2, 0};
        } else {
            err = "line " + std::to_string(p.line) +
                  ": more than two right-hand symbols (not in WCNF)";
            return -1;
        }
    }
    for (const auto &t : bin) {
        g.bin_c.push_back(std::get<0>(t));
        g.bin_a.push_back(std::get<1>(t));
        g.bin_b.push_back(std::get<2>(t));
        const auto &fm = famof[t];
        g.bin_fam.push_back(fm.first >= 0 ? fm.first : -1);
        g.bin_member.push_back(fm.second);
    }
    g.fam_size = fam_size;
    for (const auto &u : unit) {
        g.unit_c.push_back(u.first);
        g.unit_a.push_back(u.second);
    }
    g.eps.assign(eps.begin(), eps.end());
    for (auto &v : g.term_nts) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    if (g.nts.empty()) {
        err = "grammar has no productions";
        return -1;
    }
    return 0;
}

}  // namespace cflr
