// msa_io.cu -- reading aligned protein families into the int8 MSA the
// solver takes (host code).
//
// The paper's alignments are PFAM families (Sec. 4): match states are
// upper-case one-letter amino-acid codes (appendix table) or '-' (a
// deletion); insert states, which the profile HMM does not align, appear
// as lower-case letters or '.', and are removed before DCA (Sec. 4).
// States: 0 = gap ('-'), 1..20 = A C D E F G H I K L M N P Q R S T V W Y;
// the other codes of the appendix table (O, U) and the ambiguity codes
// B, Z, X are read as the gap state.  Formats: aligned FASTA / A2M
// ('>' header lines, sequence lines until the next header) and Stockholm
// ('# STOCKHOLM' header, "name sequence" lines, possibly in several
// blocks, '#' annotation lines, '//' end).
#include <cctype>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "plmdca.h"

namespace plm {
void set_error(plm_ctx *c, const char *msg);  // plm_abi.cu
}

namespace {

// -1: insert (removed), -2: not an alignment character, else the state
int state_of(unsigned char c)
{
    static const char *order = "ACDEFGHIKLMNPQRSTVWY";
    if (c == '-') return 0;
    if (c == '.' || std::islower(c)) return -1;
    if (c == 'O' || c == 'U' || c == 'B' || c == 'Z' || c == 'X') return 0;
    const char *p = std::strchr(order, c);
    if (c && p) return 1 + (int)(p - order);
    return -2;
}

struct Parsed {
    std::vector<std::vector<int8_t>> rows;
    std::string err;
};

bool append_seq(std::vector<int8_t> &row, const char *s, size_t n, std::string &err)
{
    for (size_t k = 0; k < n; ++k) {
        const unsigned char c = (unsigned char)s[k];
        if (std::isspace(c)) continue;
        const int st = state_of(c);
        if (st == -2) {
            err = std::string("unexpected character '") + (char)c + "' in a sequence";
            return false;
        }
        if (st >= 0) row.push_back((int8_t)st);
    }
    return true;
}

std::vector<std::string> lines_of(const char *text, size_t len)
{
    std::vector<std::string> out;
    size_t a = 0;
    while (a < len) {
        size_t b = a;
        while (b < len && text[b] != '\n') ++b;
        std::string ln(text + a, b - a);
        if (!ln.empty() && ln.back() == '\r') ln.pop_back();
        out.push_back(ln);
        a = b + 1;
    }
    return out;
}

bool parse_fasta(const std::vector<std::string> &lines, Parsed &P)
{
    bool in = false;
    for (const auto &ln : lines) {
        if (!ln.empty() && ln[0] == '>') {
            P.rows.emplace_back();
            in = true;
            continue;
        }
        if (!in) {
            bool blank = true;
            for (char c : ln) blank = blank && std::isspace((unsigned char)c);
            if (blank) continue;
            P.err = "sequence data before the first '>' header";
            return false;
        }
        if (!append_seq(P.rows.back(), ln.data(), ln.size(), P.err)) return false;
    }
    return true;
}

bool parse_stockholm(const std::vector<std::string> &lines, Parsed &P)
{
    std::map<std::string, size_t> index;  // name -> row, in order of first appearance
    for (const auto &ln : lines) {
        size_t a = 0;
        while (a < ln.size() && std::isspace((unsigned char)ln[a])) ++a;
        if (a == ln.size() || ln[a] == '#') continue;
        if (ln.compare(a, 2, "//") == 0) break;
        size_t b = a;
        while (b < ln.size() && !std::isspace((unsigned char)ln[b])) ++b;
        const std::string name = ln.substr(a, b - a);
        auto it = index.find(name);
        if (it == index.end()) {
            it = index.emplace(name, P.rows.size()).first;
            P.rows.emplace_back();
        }
        if (!append_seq(P.rows[it->second], ln.data() + b, ln.size() - b, P.err)) return false;
    }
    return true;
}

}  // namespace

extern "C" plm_status msa_parse(plm_ctx *ctx, const char *text, size_t len, int format,
                                int8_t *msa_out, long long capacity, int *B_out, int *N_out)
{
    auto bad = [&](const std::string &m) {
        plm::set_error(ctx, m.c_str());
        return PLM_EINVAL;
    };
    if (!text || !B_out || !N_out) return bad("text, B_out and N_out are required");
    *B_out = 0;
    *N_out = 0;
    std::vector<std::string> lines = lines_of(text, len);
    if (format == 0) {
        // auto: Stockholm if its header comes first, else FASTA
        format = 1;
        for (const auto &ln : lines) {
            if (ln.empty()) continue;
            if (ln.compare(0, 11, "# STOCKHOLM") == 0) format = 2;
            break;
        }
    }
    Parsed P;
    bool ok;
    if (format == 1) ok = parse_fasta(lines, P);
    else if (format == 2) ok = parse_stockholm(lines, P);
    else return bad("format must be 0 (auto), 1 (FASTA) or 2 (Stockholm)");
    if (!ok) return bad(P.err);
    if (P.rows.empty()) return bad("no sequences");
    const size_t N = P.rows[0].size();
    for (size_t b = 0; b < P.rows.size(); ++b)
        if (P.rows[b].size() != N)
            return bad("sequence " + std::to_string(b) + " has " +
                       std::to_string(P.rows[b].size()) + " match columns, the first has " +
                       std::to_string(N));
    if (N == 0 || P.rows.size() > 0x7fffffff || N > 0x7fffffff)
        return bad("no match columns, or too large");
    *B_out = (int)P.rows.size();
    *N_out = (int)N;
    if (!msa_out) return PLM_OK;
    if (capacity < (long long)(P.rows.size() * N)) return bad("capacity is less than B * N");
    for (size_t b = 0; b < P.rows.size(); ++b) std::memcpy(msa_out + b * N, P.rows[b].data(), N);
    return PLM_OK;
}
