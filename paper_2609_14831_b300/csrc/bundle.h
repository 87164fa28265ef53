// bundle.h -- on-disk form of a compiled operation graph (paper Sec. 2.3:
// the saved bundle records the registry, block mask, factor table and
// identifiers, so that it can be checked and reloaded in another process).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace cut {

// Packed record: w0 = (code << 24) | in1, w1 = in2.  Indices < 2^24.
constexpr uint32_t kIndexBits = 24;
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1;
constexpr int kMaxCodes = 256;

struct Sha256 {
    uint32_t h[8];
    uint64_t len = 0;
    uint8_t buf[64];
    size_t nbuf = 0;
    Sha256();
    void update(const void *data, size_t n);
    void final(uint8_t out[32]);
    static void digest(const void *data, size_t n, uint8_t out[32]);
};

// In-memory graph (host).  Stage 0 = generator (rows: generator coordinate
// a; inputs i = diagonal coordinate, j = off-diagonal coordinate).  Stage 1 =
// commutator (rows: output coordinate k; inputs a, j).  Stage 2 = optional
// outside-space records (rows: labels outside the registry, inputs a, j).
struct HostGraph {
    int algebra = 0, nmodes = 0, max_rank = 0;
    std::vector<uint64_t> labels;      // [n]
    std::vector<uint64_t> gen_labels;  // [n_g]
    std::vector<uint64_t> out_labels;  // [n_out] outside-space labels (diagnostics)
    std::vector<uint8_t> diag;         // [n]
    std::vector<int32_t> num, den;     // factor table
    std::vector<uint64_t> rp[3];       // row pointers
    std::vector<uint32_t> rec[3];      // 2 words per record
    uint8_t sha[32] = {0};
    int64_t n() const { return (int64_t)labels.size(); }
    int64_t n_g() const { return (int64_t)gen_labels.size(); }
    int64_t n_out() const { return (int64_t)out_labels.size(); }
    int64_t R(int s) const { return (int64_t)(rec[s].size() / 2); }
};

// Write a bundle; computes and stores the payload digest.  Returns "" or an
// error message.
std::string write_bundle(HostGraph &g, const std::string &path, int64_t *bytes);
// Read and validate.  Returns 0 (ok), 2 (io), 3 (format), 4 (checksum);
// message in *err.
int read_bundle(const std::string &path, HostGraph &g, std::string *err);

}  // namespace cut
