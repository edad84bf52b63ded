// Test helper: run the library's grammar compiler on the text read from
// standard input and print its tables as JSON, by symbol name (the Python
// side compares them with the oracle's independent reader).
#include "grammar.h"

#include <cstdio>
#include <iostream>
#include <iterator>
#include <string>

static void names(const cflr::Grammar &g, const std::vector<uint32_t> &ids) {
    std::printf("[");
    for (size_t i = 0; i < ids.size(); i++) std::printf("%s\"%s\"", i ? "," : "", g.nts[ids[i]].c_str());
    std::printf("]");
}

int main() {
    std::string text((std::istreambuf_iterator<char>(std::cin)), std::istreambuf_iterator<char>());
    cflr::Grammar g;
    std::string err;
    if (cflr::parse_grammar(text.data(), text.size(), g, err) != 0) {
        std::printf("{\"error\": \"parse failed\"}\n");
        return 0;
    }
    std::printf("{\"n_named\": %u, \"nts\": [", g.n_named);
    for (size_t i = 0; i < g.nts.size(); i++) std::printf("%s\"%s\"", i ? "," : "", g.nts[i].c_str());
    std::printf("], \"binary\": [");
    for (size_t p = 0; p < g.bin_c.size(); p++)
        std::printf("%s[\"%s\",\"%s\",\"%s\",%d,%u]", p ? "," : "", g.nts[g.bin_c[p]].c_str(),
                    g.nts[g.bin_a[p]].c_str(), g.nts[g.bin_b[p]].c_str(), (int)g.bin_fam[p],
                    g.bin_member[p]);
    std::printf("], \"fam_size\": [");
    for (size_t f = 0; f < g.fam_size.size(); f++) std::printf("%s%u", f ? "," : "", g.fam_size[f]);
    std::printf("], \"unit\": [");
    for (size_t p = 0; p < g.unit_c.size(); p++)
        std::printf("%s[\"%s\",\"%s\"]", p ? "," : "", g.nts[g.unit_c[p]].c_str(),
                    g.nts[g.unit_a[p]].c_str());
    std::printf("], \"eps\": ");
    names(g, g.eps);
    std::printf(", \"term\": {");
    for (size_t t = 0; t < g.terms.size(); t++) {
        std::printf("%s\"%s\": ", t ? "," : "", g.terms[t].c_str());
        names(g, g.term_nts[t]);
    }
    std::printf("}}\n");
    return 0;
}
