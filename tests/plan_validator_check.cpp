// The plan check (validate_plan) on a real plan and on five corruptions of
// it, one per kind of index the device kernels use: a near-list leaf out of
// range, non-monotone near pointers, a wrong entry count, an interaction
// entry naming a cluster out of range and one naming a translation row out
// of range.  Reads an icosphere's nodes and triangles from the two files
// named on the command line (float64 [n_nodes, 3], int32 [n_tris, 3]) and
// prints one line per case: its name and the check's message ("ok" if none).
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../paper_2312_00005_gb300/csrc/bem_plan.hpp"

using namespace bem;

template <typename T>
static std::vector<T> read_all(const char *path)
{
    std::vector<T> v;
    FILE *f = std::fopen(path, "rb");
    if (!f) return v;
    std::fseek(f, 0, SEEK_END);
    const long nb = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    v.resize((size_t)nb / sizeof(T));
    if (std::fread(v.data(), sizeof(T), v.size(), f) != v.size()) v.clear();
    std::fclose(f);
    return v;
}

static void report(const char *name, const std::string &msg) { std::printf("%s: %s\n", name, msg.empty() ? "ok" : msg.c_str()); }

int main(int argc, char **argv)
{
    if (argc < 3) return 2;
    const std::vector<double> nodes = read_all<double>(argv[1]);
    const std::vector<int32_t> tris = read_all<int32_t>(argv[2]);
    if (nodes.empty() || tris.empty()) return 2;
    bem_params p;
    bem_params_default(&p);
    Geometry g;
    if (!compute_geometry(nodes.data(), (int64_t)nodes.size() / 3, tris.data(), (int64_t)tris.size() / 3, g).empty())
        return 2;
    Tree t;
    build_tree(g, auto_leaf_edge(g, p), t);
    FreqPlan fp;
    build_plan(g, t, p, 2.0 * M_PI * 3000.0 / 343.0, fp);
    report("valid", validate_plan(t, fp));
    if (fp.far.empty() || fp.far[0].il_src.empty() || fp.near_src.size() < 2) return 3;
    const int nl = (int)fp.near_ptr.size() - 1;
    {
        FreqPlan b = fp;
        b.near_src[0] = nl;
        report("near_leaf_out_of_range", validate_plan(t, b));
    }
    {
        FreqPlan b = fp;
        b.near_ptr[1] = b.near_ptr[2] + 1;
        report("near_pointers_not_monotone", validate_plan(t, b));
    }
    {
        FreqPlan b = fp;
        b.nnz += 1;
        report("entry_count", validate_plan(t, b));
    }
    {
        FreqPlan b = fp;
        b.far[0].il_src[0] = b.far[0].nc;
        report("cluster_out_of_range", validate_plan(t, b));
    }
    {
        FreqPlan b = fp;
        b.far[0].il_off[0] = (int32_t)(b.far[0].offsets.size() / 3);
        report("translation_row_out_of_range", validate_plan(t, b));
    }
    return 0;
}
