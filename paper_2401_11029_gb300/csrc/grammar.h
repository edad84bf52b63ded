// Grammar compiler of the CUDA library (host C++).
//
// Reads the WCNF text format declared in include/cflr.h and produces the
// tables the device loop needs: binary productions (c, a, b), unit
// productions (c, a), epsilon non-terminals, and for every terminal the
// non-terminals that derive it directly.  Paper Sec. 2 (WCNF definition)
// and appendix B (indexed non-terminals, hand-made WCNF grammars).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace cflr {

struct Grammar {
    std::vector<std::string> nts;        // non-terminal names; wrappers "<x>" last
    uint32_t n_named = 0;                // non-terminals named in the text
    std::vector<std::string> terms;      // terminal names (edge labels)
    std::vector<uint32_t> bin_c, bin_a, bin_b;   // c -> a b
    // Indexed families (appendix B; optimisation 4): a production line with
    // one index variable of range size F >= 2 expands to F members.  For each
    // binary production: its family (-1: none) and member index 0..F-1.
    std::vector<int32_t> bin_fam;
    std::vector<uint32_t> bin_member;
    std::vector<uint32_t> fam_size;              // family id -> F
    std::vector<uint32_t> unit_c, unit_a;        // c -> a
    std::vector<uint32_t> eps;                   // A -> eps
    std::vector<std::vector<uint32_t>> term_nts; // terminal id -> {A | A -> x}

    int find_nt(const std::string &s) const;
    int find_term(const std::string &s) const;
};

// Returns 0 on success; on failure a message naming the line in err.
int parse_grammar(const char *text, size_t len, Grammar &g, std::string &err);

}  // namespace cflr
