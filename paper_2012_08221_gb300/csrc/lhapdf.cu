// Reader of LHAPDF "lhagrid1" PDF sets (host only; no GPU involved).
//
// The paper keeps the community grid format and folder layout (PDFFlow
// Sec. 1 and Sec. 4): a set is a folder <name>/ holding <name>.info (YAML
// metadata) and one <name>_<mmmm>.dat file per member.  A member file has a
// header ending in a line "---", then one block per Q subgrid, each block
//   line 1: x knots;  line 2: Q knots (GeV);  line 3: PDG ids;
//   then n_x * n_q lines of n_flav values of x*f, x knot outer, Q knot inner,
// and each block is closed by a line "---".  Consecutive subgrids share their
// boundary Q knot.  The reader fills a pdfgpu_grid_desc whose arrays it owns.
#include <ctype.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "pdf_internal.h"

using namespace pdfgpu;

struct pdfgpu_lhapdf {
    std::vector<double> x, q, values, alphas;
    std::vector<int32_t> nq, pids;
    int32_t n_members = 0;
    bool has_alphas = false;
};

namespace {

std::string trim(const std::string &s)
{
    size_t a = 0, b = s.size();
    while (a < b && isspace((unsigned char)s[a])) ++a;
    while (b > a && isspace((unsigned char)s[b - 1])) --b;
    return s.substr(a, b - a);
}

bool parse_numbers(const std::string &line, std::vector<double> &out)
{
    out.clear();
    const char *p = line.c_str();
    char *end = nullptr;
    while (*p) {
        while (*p && (isspace((unsigned char)*p) || *p == ',' || *p == '[' || *p == ']')) ++p;
        if (!*p) break;
        double v = strtod(p, &end);
        if (end == p) return false;
        out.push_back(v);
        p = end;
    }
    return true;
}

// Number(s) of a key: a scalar, or a flow-style YAML list "[a, b, c]"
// possibly continued on the following lines until the closing bracket.
bool info_list(const std::string &text, const std::string &key, std::vector<double> &out)
{
    std::istringstream in(text);
    std::string line;
    while (std::getline(in, line)) {
        std::string t = trim(line);
        if (t.compare(0, key.size() + 1, key + ":") != 0) continue;
        std::string rest = t.substr(key.size() + 1);
        if (rest.find('[') != std::string::npos)
            while (rest.find(']') == std::string::npos && std::getline(in, line)) rest += " " + line;
        return parse_numbers(rest, out);
    }
    return false;
}

struct Member {
    std::vector<double> x, q;
    std::vector<int32_t> nq, pids;
    std::vector<std::vector<double>> blocks;  // per subgrid: [ix][iq][flav]
};

int read_member(const std::string &path, Member &m)
{
    std::ifstream f(path);
    if (!f) return fail(PDF_E_ARG, "cannot open " + path);
    std::string line;
    bool header = true, format_ok = false;
    std::vector<double> nums;
    while (std::getline(f, line)) {
        std::string t = trim(line);
        if (header) {
            if (t == "---") {
                header = false;
                continue;
            }
            if (t.rfind("Format:", 0) == 0 && t.find("lhagrid1") != std::string::npos) format_ok = true;
            continue;
        }
        if (t.empty()) continue;
        // a subgrid block starts: x knots, Q knots, pids
        std::vector<double> xs, qs, ps;
        if (!parse_numbers(t, xs) || xs.size() < 2) return fail(PDF_E_DESC, path + ": bad x knot line");
        if (!std::getline(f, line) || !parse_numbers(line, qs) || qs.size() < 2)
            return fail(PDF_E_DESC, path + ": bad Q knot line");
        if (!std::getline(f, line) || !parse_numbers(line, ps) || ps.empty())
            return fail(PDF_E_DESC, path + ": bad flavour line");
        if (m.x.empty()) {
            m.x = xs;
            for (double p : ps) m.pids.push_back((int32_t)p);
        } else {
            if (xs != m.x) return fail(PDF_E_DESC, path + ": subgrids with different x knots");
            if (ps.size() != m.pids.size()) return fail(PDF_E_DESC, path + ": subgrids with different flavours");
        }
        const size_t nx = xs.size(), nqs = qs.size(), nf = ps.size();
        std::vector<double> block(nx * nqs * nf);
        for (size_t l = 0; l < nx * nqs; ++l) {
            if (!std::getline(f, line) || !parse_numbers(line, nums) || nums.size() != nf)
                return fail(PDF_E_DESC, path + ": bad value line");
            std::copy(nums.begin(), nums.end(), block.begin() + l * nf);
        }
        if (!std::getline(f, line) || trim(line) != "---")
            return fail(PDF_E_DESC, path + ": subgrid block not closed by ---");
        m.q.insert(m.q.end(), qs.begin(), qs.end());
        m.nq.push_back((int32_t)nqs);
        m.blocks.push_back(std::move(block));
    }
    if (!format_ok) return fail(PDF_E_DESC, path + ": not an lhagrid1 file");
    if (m.blocks.empty()) return fail(PDF_E_DESC, path + ": no subgrid");
    return PDF_OK;
}

}  // namespace

extern "C" int pdf_lhapdf_open(const char *set_dir, int32_t first_member, int32_t n_members,
                               pdfgpu_lhapdf_t *out)
{
    PDF_TRACE("pdf_lhapdf_open");
    clear_error();
    if (!set_dir || !out || first_member < 0 || n_members < 1) return fail(PDF_E_ARG, "bad argument");
    *out = nullptr;
    std::string dir(set_dir);
    while (dir.size() > 1 && dir.back() == '/') dir.pop_back();
    std::string name = dir.substr(dir.find_last_of('/') + 1);
    std::string info_text;
    {
        std::ifstream f(dir + "/" + name + ".info");
        if (!f) return fail(PDF_E_ARG, "cannot open " + dir + "/" + name + ".info");
        std::stringstream ss;
        ss << f.rdbuf();
        info_text = ss.str();
    }
    std::vector<double> num;
    if (info_list(info_text, "NumMembers", num) && !num.empty() && first_member + n_members > (int)num[0])
        return fail(PDF_E_RANGE, "members beyond NumMembers of the set");
    pdfgpu_lhapdf *h = new pdfgpu_lhapdf();
    for (int k = 0; k < n_members; ++k) {
        char buf[32];
        snprintf(buf, sizeof buf, "_%04d.dat", first_member + k);
        Member m;
        int rc = read_member(dir + "/" + name + buf, m);
        if (rc) {
            delete h;
            return rc;
        }
        if (k == 0) {
            h->x = m.x;
            h->q = m.q;
            h->nq = m.nq;
            h->pids = m.pids;
        } else if (m.x != h->x || m.q != h->q || m.nq != h->nq || m.pids != h->pids) {
            delete h;
            return fail(PDF_E_DESC, "members with different knots or flavours");
        }
        // [ix][iq][flav] per subgrid -> [row][ix][flav] of the member
        const size_t nx = h->x.size(), nf = h->pids.size();
        size_t r0 = 0;
        size_t base = h->values.size();
        h->values.resize(base + h->q.size() * nx * nf);
        for (size_t s = 0; s < m.blocks.size(); ++s) {
            const size_t nqs = (size_t)m.nq[s];
            for (size_t ix = 0; ix < nx; ++ix)
                for (size_t iq = 0; iq < nqs; ++iq)
                    for (size_t a = 0; a < nf; ++a)
                        h->values[base + ((r0 + iq) * nx + ix) * nf + a] = m.blocks[s][(ix * nqs + iq) * nf + a];
            r0 += nqs;
        }
    }
    h->n_members = n_members;
    // alpha_s knots: attached when they are the grid's own Q knots
    std::vector<double> aq, av;
    if (info_list(info_text, "AlphaS_Qs", aq) && info_list(info_text, "AlphaS_Vals", av) &&
        aq.size() == av.size() && aq == h->q) {
        h->alphas = av;
        h->has_alphas = true;
    }
    *out = h;
    return PDF_OK;
}

extern "C" int pdf_lhapdf_desc(pdfgpu_lhapdf_t h, pdfgpu_grid_desc *desc)
{
    PDF_TRACE("pdf_lhapdf_desc");
    clear_error();
    if (!h || !desc) return fail(PDF_E_ARG, "null argument");
    memset(desc, 0, sizeof(*desc));
    desc->n_x = (int32_t)h->x.size();
    desc->x_knots = h->x.data();
    desc->n_sub = (int32_t)h->nq.size();
    desc->n_q = h->nq.data();
    desc->q_knots = h->q.data();
    desc->n_flav = (int32_t)h->pids.size();
    desc->pids = h->pids.data();
    desc->n_members = h->n_members;
    desc->values = h->values.data();
    desc->alphas = h->has_alphas ? h->alphas.data() : nullptr;
    desc->interp = PDF_INTERP_LOGBICUBIC;
    desc->extrap = PDF_EXTRAP_LINEAR;
    return PDF_OK;
}

extern "C" int pdf_lhapdf_close(pdfgpu_lhapdf_t h)
{
    PDF_TRACE("pdf_lhapdf_close");
    clear_error();
    if (!h) return fail(PDF_E_ARG, "null handle");
    delete h;
    return PDF_OK;
}
