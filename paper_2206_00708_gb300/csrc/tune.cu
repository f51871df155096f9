// Launch-shape table of the autotuner: for each tuned kernel family, problem width
// (columns per launch) and size class (ceil(log2(rows))), the thread-block size and
// kernel variant that ran fastest when bem_autotune timed the candidates on this GPU.
// Kernels look their shape up here and fall back to their built-in defaults when no
// entry exists.  The table can be saved to and loaded from a small JSON file, so a
// tuning run on one GB300 serves later processes on the same kind of GPU.
#include "bem_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <sstream>
#include <stdexcept>
#include <string>
#include <vector>

namespace bem {

namespace {

struct TuneEntry {
    int kernel, width, nlog2;
    TuneChoice c;
};

std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

const char* const kNames[TUNE_KERNELS] = {"gemm_tc", "cheb"};

int kernel_id(const std::string& name) {
    for (int k = 0; k < TUNE_KERNELS; ++k)
        if (name == kNames[k]) return k;
    return -1;
}

// value of "key": <number> or "key": "<string>" inside one JSON object (flat, as written
// by bem_tune_save); false when absent
bool json_field(const std::string& obj, const char* key, std::string& out) {
    const std::string pat = std::string("\"") + key + "\"";
    size_t p = obj.find(pat);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + pat.size());
    if (p == std::string::npos) return false;
    ++p;
    while (p < obj.size() && (obj[p] == ' ' || obj[p] == '\t' || obj[p] == '\n' || obj[p] == '\r')) ++p;
    if (p >= obj.size()) return false;
    if (obj[p] == '"') {
        const size_t e = obj.find('"', p + 1);
        if (e == std::string::npos) return false;
        out = obj.substr(p + 1, e - p - 1);
        return true;
    }
    size_t e = p;
    while (e < obj.size() && (std::isdigit((unsigned char)obj[e]) || obj[e] == '-' || obj[e] == '.' || obj[e] == 'e' ||
                              obj[e] == 'E' || obj[e] == '+'))
        ++e;
    if (e == p) return false;
    out = obj.substr(p, e - p);
    return true;
}

}  // namespace

int size_class(int64_t n) {
    int c = 0;
    while (c < 62 && ((int64_t)1 << c) < n) ++c;
    return c;
}

TuneChoice tune_get(int kernel, int width, int64_t n, TuneChoice dflt) {
    const int nl = size_class(n);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry& e : g_tune)
        if (e.kernel == kernel && e.width == width && e.nlog2 == nl) return e.c;
    return dflt;
}

void tune_put(int kernel, int width, int64_t n, TuneChoice c) {
    const int nl = size_class(n);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (TuneEntry& e : g_tune)
        if (e.kernel == kernel && e.width == width && e.nlog2 == nl) {
            e.c = c;
            return;
        }
    g_tune.push_back({kernel, width, nl, c});
}

}  // namespace bem

using namespace bem;

extern "C" {

void bem_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

int32_t bem_tune_count(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int32_t)g_tune.size();
}

bem_status bem_tune_get(const char* kernel, int32_t width, int64_t rows, int32_t* block, int32_t* variant,
                        double* ms) {
    BEM_REQUIRE(kernel != nullptr && block != nullptr && variant != nullptr, "null argument");
    const int k = kernel_id(kernel);
    BEM_REQUIRE(k >= 0, std::string("unknown tuned kernel ") + kernel);
    const TuneChoice none{0, 0, 0.0};
    const TuneChoice c = tune_get(k, width, rows, none);
    *block = c.block;
    *variant = c.variant;
    if (ms) *ms = c.ms;
    return BEM_OK;
}

bem_status bem_tune_save(const char* path) {
    BEM_REQUIRE(path != nullptr, "null path");
    std::ostringstream os;
    os << "{\"format\": \"bem-tune-1\", \"entries\": [\n";
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (size_t i = 0; i < g_tune.size(); ++i) {
            const TuneEntry& e = g_tune[i];
            char line[256];
            std::snprintf(line, sizeof line,
                          "  {\"kernel\": \"%s\", \"width\": %d, \"n_log2\": %d, \"block\": %d, \"variant\": %d, "
                          "\"ms\": %.6g}%s\n",
                          kNames[e.kernel], e.width, e.nlog2, e.c.block, e.c.variant, e.c.ms,
                          i + 1 < g_tune.size() ? "," : "");
            os << line;
        }
    }
    os << "]}\n";
    FILE* f = std::fopen(path, "w");
    if (!f) {
        set_error(std::string("cannot open ") + path + " for writing");
        return BEM_E_INVALID_ARG;
    }
    const std::string s = os.str();
    const size_t w = std::fwrite(s.data(), 1, s.size(), f);
    std::fclose(f);
    if (w != s.size()) {
        set_error(std::string("short write to ") + path);
        return BEM_E_INTERNAL;
    }
    return BEM_OK;
}

bem_status bem_tune_load(const char* path) {
    BEM_REQUIRE(path != nullptr, "null path");
    FILE* f = std::fopen(path, "r");
    if (!f) {
        set_error(std::string("cannot open ") + path);
        return BEM_E_INVALID_ARG;
    }
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, r);
    std::fclose(f);
    BEM_REQUIRE(text.find("\"bem-tune-1\"") != std::string::npos, "not a bem tuning file (format bem-tune-1)");
    const size_t arr = text.find('[');
    BEM_REQUIRE(arr != std::string::npos, "tuning file has no entries array");
    std::vector<TuneEntry> got;
    size_t p = arr;
    while ((p = text.find('{', p)) != std::string::npos) {
        const size_t e = text.find('}', p);
        BEM_REQUIRE(e != std::string::npos, "unterminated entry in tuning file");
        const std::string obj = text.substr(p, e - p + 1);
        std::string name, w, nl, b, v, ms;
        BEM_REQUIRE(json_field(obj, "kernel", name) && json_field(obj, "width", w) && json_field(obj, "n_log2", nl) &&
                        json_field(obj, "block", b) && json_field(obj, "variant", v),
                    "tuning entry misses a field");
        const int k = kernel_id(name);
        BEM_REQUIRE(k >= 0, "unknown kernel in tuning file: " + name);
        TuneEntry t{k, 0, 0, {0, 0, 0.0}};
        try {  // numbers as written by bem_tune_save; anything else is a malformed file
            t.width = std::stoi(w);
            t.nlog2 = std::stoi(nl);
            t.c.block = std::stoi(b);
            t.c.variant = std::stoi(v);
            if (json_field(obj, "ms", ms)) t.c.ms = std::stod(ms);
        } catch (const std::exception&) {
            set_error("tuning entry holds a malformed number");
            return BEM_E_INVALID_ARG;
        }
        BEM_REQUIRE(t.width >= 1 && t.width <= 256 && t.nlog2 >= 0 && t.nlog2 <= 62, "tuning entry out of range");
        BEM_REQUIRE(tune_choice_valid(k, t.c), "tuning entry names an unsupported block size or variant");
        got.push_back(t);
        p = e + 1;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry& t : got) {
        bool found = false;
        for (TuneEntry& e : g_tune)
            if (e.kernel == t.kernel && e.width == t.width && e.nlog2 == t.nlog2) {
                e = t;
                found = true;
            }
        if (!found) g_tune.push_back(t);
    }
    return BEM_OK;
}

}  // extern "C"

namespace {
// A tuning file named by the environment variable BEM_TUNE_FILE is merged into the table
// when the library is loaded, so that shapes tuned once serve every later process.  A
// missing or malformed file leaves the table empty (nothing else changes).
struct TuneFileAtLoad {
    TuneFileAtLoad() {
        const char* path = std::getenv("BEM_TUNE_FILE");
        if (path && *path) bem_tune_load(path);
    }
} g_tune_file_at_load;
}  // namespace
