// tune.cu — autotuner of the H-matvec launch parameters (no paper
// counterpart: the shapes of the persistent product kernels are picked per
// GPU and per workload class by measurement).
//
// Tuned parameters (matvec_set_params):
//   BF16 storage: the number of shared-memory stages of the streamed product
//                 kernels (2, 3 or 4 rings of 12 KB; 4 leaves room for three
//                 CTAs per SM instead of four);
//   FP32 storage: the byte size of a work item (128 KB .. 1 MB): smaller items
//                 balance the grid, larger ones amortise the per-item setup.
// Each candidate is timed on the handle itself (CUDA events around repeated
// products on the handle's work vectors, after warm-up); the fastest wins.
// Results are kept in a text cache file, one line per key:
//   hm-tune-1 <key> nstage=<n> item_bytes=<b> ms=<best ms>
// with key = GPU name, storage, largest leading dimension of the stored
// chunks, and log2 of the product's algorithmic bytes (the workload class).
// A build that finds its key applies the cached parameters without timing;
// one that does not runs the sweep and writes the line (the file is rewritten
// through a temporary and renamed).  Malformed lines are ignored.  The tuned
// parameters change only how the work is scheduled, never what is summed.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "hm_internal.h"
#include "matvec_dev.cuh"

namespace {

std::string tune_key(hm_matrix* h) {
    cudaDeviceProp prop;
    HM_CUDA(cudaGetDeviceProperties(&prop, h->device));
    std::string gpu = prop.name;
    for (char& c : gpu)
        if (c == ' ' || c == '\t') c = '_';
    int ldmax = 0;
    for (const Chunk& c : h->plan.chunks) ldmax = std::max(ldmax, (int)c.ld);
    int64_t alg[3];
    matvec_alg_bytes(h->mv, 3 * h->nc, alg);
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= alg[2]) ++lg;
    std::ostringstream k;
    k << "gpu=" << gpu << ";storage=" << (h->opts.storage == HM_STORE_BF16 ? "bf16" : "fp32")
      << ";ld=" << ldmax << ";log2bytes=" << lg;
    return k.str();
}

struct Entry {
    int nstage = 3;
    int64_t item_bytes = 256 * 1024;
    double ms = 0;
};

bool parse_line(const std::string& line, std::string& key, Entry& e) {
    std::istringstream is(line);
    std::string tag, f1, f2, f3;
    if (!(is >> tag >> key >> f1 >> f2 >> f3) || tag != "hm-tune-1") return false;
    if (f1.rfind("nstage=", 0) || f2.rfind("item_bytes=", 0) || f3.rfind("ms=", 0)) return false;
    char* end = nullptr;
    const long ns = std::strtol(f1.c_str() + 7, &end, 10);
    if (*end) return false;
    const long long ib = std::strtoll(f2.c_str() + 11, &end, 10);
    if (*end) return false;
    const double ms = std::strtod(f3.c_str() + 3, &end);
    if (*end) return false;
    if (ns < 2 || ns > 4 || ib < 16 * 1024 || ib > 16 * 1024 * 1024 || !(ms >= 0)) return false;
    e.nstage = (int)ns;
    e.item_bytes = ib;
    e.ms = ms;
    return true;
}

std::vector<std::string> read_lines(const char* path) {
    std::vector<std::string> out;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) out.push_back(line);
    return out;
}

void write_entry(const char* path, const std::string& key, const Entry& e) {
    std::vector<std::string> lines = read_lines(path);
    std::ostringstream l;
    l << "hm-tune-1 " << key << " nstage=" << e.nstage << " item_bytes=" << e.item_bytes
      << " ms=" << e.ms;
    bool replaced = false;
    for (std::string& s : lines) {
        std::string k;
        Entry old;
        if (parse_line(s, k, old) && k == key) {
            s = l.str();
            replaced = true;
        }
    }
    if (!replaced) lines.push_back(l.str());
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) hm_throw(HM_ERR_ARG, std::string("cannot write the tune cache ") + tmp);
        for (const std::string& s : lines) f << s << "\n";
        if (!f) hm_throw(HM_ERR_ARG, std::string("cannot write the tune cache ") + tmp);
    }
    if (std::rename(tmp.c_str(), path) != 0)
        hm_throw(HM_ERR_ARG, std::string("cannot replace the tune cache ") + path);
}

// mean device ms of one product with the current parameters
double time_product(hm_matrix* h, cudaStream_t st, int reps) {
    const int64_t ndof = 3 * h->nc;
    if (!h->d_xp || !h->d_yp || !h->mv) hm_throw(HM_ERR_CUDA, "tuning before the work vectors exist");
    for (int r = 0; r < 2; ++r) matvec_tree_order(h->mv, h->d_xp, h->d_yp, ndof, st);
    cudaEvent_t a, b;
    HM_CUDA(cudaEventCreate(&a));
    HM_CUDA(cudaEventCreate(&b));
    HM_CUDA(cudaEventRecord(a, st));
    for (int r = 0; r < reps; ++r) matvec_tree_order(h->mv, h->d_xp, h->d_yp, ndof, st);
    HM_CUDA(cudaEventRecord(b, st));
    HM_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    HM_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (matvec_take_error(h->mv, st))
        hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies (tuning)");
    return ms / reps;
}

}  // namespace

void tune_product(hm_matrix* h, const char* path, cudaStream_t st) {
    h->tune_source = "default";
    if (!path || !*path) return;
    const std::string key = tune_key(h);
    for (const std::string& line : read_lines(path)) {
        std::string k;
        Entry e;
        if (parse_line(line, k, e) && k == key) {
            matvec_set_params(h->mv, h->plan, e.nstage, e.item_bytes, st);
            h->tune_source = "cache";
            h->tune_nstage = e.nstage;
            h->tune_item_bytes = e.item_bytes;
            h->tune_ms = e.ms;
            h->tune_key = key;
            return;
        }
    }
    std::vector<Entry> cand;
    if (h->opts.storage == HM_STORE_BF16) {
        for (int ns : {2, 3, 4}) cand.push_back({ns, h->mv->item_bytes, 0});
    } else {
        for (int64_t ib : {128 * 1024, 256 * 1024, 512 * 1024, 1024 * 1024})
            cand.push_back({h->mv->s16_nstage, ib, 0});
    }
    std::ostringstream trials;
    Entry best;
    best.ms = 1e300;
    for (Entry& e : cand) {
        matvec_set_params(h->mv, h->plan, e.nstage, e.item_bytes, st);
        e.ms = time_product(h, st, 5);
        trials << (trials.tellp() > 0 ? ", " : "") << "{\"nstage\": " << e.nstage
               << ", \"item_bytes\": " << e.item_bytes << ", \"ms\": " << e.ms << "}";
        if (e.ms < best.ms) best = e;
    }
    matvec_set_params(h->mv, h->plan, best.nstage, best.item_bytes, st);
    write_entry(path, key, best);
    h->tune_source = "sweep";
    h->tune_nstage = best.nstage;
    h->tune_item_bytes = best.item_bytes;
    h->tune_ms = best.ms;
    h->tune_key = key;
    h->tune_trials = trials.str();
}
