// bundle.cpp -- bundle file format, SHA-256 (FIPS 180-4), validated reload.
#include "bundle.h"

#include <cstdio>
#include <cstring>
#include <memory>

namespace cut {

// ---------------------------------------------------------------- SHA-256
static const uint32_t K256[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};

static inline uint32_t rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

static void sha_block(uint32_t h[8], const uint8_t *p) {
    uint32_t w[64];
    for (int t = 0; t < 16; t++)
        w[t] = (uint32_t)p[4 * t] << 24 | (uint32_t)p[4 * t + 1] << 16 | (uint32_t)p[4 * t + 2] << 8 |
               (uint32_t)p[4 * t + 3];
    for (int t = 16; t < 64; t++) {
        uint32_t s0 = rotr(w[t - 15], 7) ^ rotr(w[t - 15], 18) ^ (w[t - 15] >> 3);
        uint32_t s1 = rotr(w[t - 2], 17) ^ rotr(w[t - 2], 19) ^ (w[t - 2] >> 10);
        w[t] = w[t - 16] + s0 + w[t - 7] + s1;
    }
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
    for (int t = 0; t < 64; t++) {
        uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t t1 = hh + S1 + ch + K256[t] + w[t];
        uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
        uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t t2 = S0 + mj;
        hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
    }
    h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

Sha256::Sha256() {
    const uint32_t init[8] = {0x6a09e667, 0xbb67ae85, 0x3c6ef372, 0xa54ff53a,
                              0x510e527f, 0x9b05688c, 0x1f83d9ab, 0x5be0cd19};
    memcpy(h, init, sizeof(h));
}

void Sha256::update(const void *data, size_t n) {
    const uint8_t *p = (const uint8_t *)data;
    len += n;
    if (nbuf) {
        size_t take = 64 - nbuf < n ? 64 - nbuf : n;
        memcpy(buf + nbuf, p, take);
        nbuf += take; p += take; n -= take;
        if (nbuf == 64) { sha_block(h, buf); nbuf = 0; }
    }
    while (n >= 64) { sha_block(h, p); p += 64; n -= 64; }
    if (n) { memcpy(buf, p, n); nbuf = n; }
}

void Sha256::final(uint8_t out[32]) {
    uint64_t bits = len * 8;
    uint8_t pad = 0x80;
    update(&pad, 1);
    uint8_t z = 0;
    while (nbuf != 56) update(&z, 1);
    uint8_t lb[8];
    for (int i = 0; i < 8; i++) lb[i] = (uint8_t)(bits >> (56 - 8 * i));
    update(lb, 8);
    for (int i = 0; i < 8; i++) {
        out[4 * i] = (uint8_t)(h[i] >> 24); out[4 * i + 1] = (uint8_t)(h[i] >> 16);
        out[4 * i + 2] = (uint8_t)(h[i] >> 8); out[4 * i + 3] = (uint8_t)h[i];
    }
}

void Sha256::digest(const void *data, size_t n, uint8_t out[32]) {
    Sha256 s;
    s.update(data, n);
    s.final(out);
}

// ---------------------------------------------------------------- format
struct FileHeader {
    char magic[8];
    uint32_t version, algebra, nmodes, max_rank;
    uint64_t n, n_g, R0, R1;
    uint32_t n_codes, reserved;
    uint64_t payload_bytes;
    uint8_t sha256[32];
    uint64_t n_out, R2;   // outside-space labels and records (0 without diagnostics)
    uint8_t pad[160 - 8 - 16 - 32 - 8 - 8 - 32 - 16];
};
static_assert(sizeof(FileHeader) == 160, "header size");
static const char kMagic[8] = {'C', 'U', 'T', 'G', 'R', 'A', 'P', 'H'};
static const uint32_t kVersion = 2;

static size_t pad64(size_t b) { return (b + 63) & ~size_t(63); }

struct Section { void *ptr; size_t bytes; };

static std::vector<Section> sections(HostGraph &g) {
    return {{g.labels.data(), g.labels.size() * 8},      {g.gen_labels.data(), g.gen_labels.size() * 8},
            {g.diag.data(), g.diag.size()},               {g.num.data(), g.num.size() * 4},
            {g.den.data(), g.den.size() * 4},             {g.rp[0].data(), g.rp[0].size() * 8},
            {g.rec[0].data(), g.rec[0].size() * 4},       {g.rp[1].data(), g.rp[1].size() * 8},
            {g.rec[1].data(), g.rec[1].size() * 4},       {g.out_labels.data(), g.out_labels.size() * 8},
            {g.rp[2].data(), g.rp[2].size() * 8},         {g.rec[2].data(), g.rec[2].size() * 4}};
}

std::string write_bundle(HostGraph &g, const std::string &path, int64_t *bytes) {
    FileHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, 8);
    hd.version = kVersion;
    hd.algebra = (uint32_t)g.algebra;
    hd.nmodes = (uint32_t)g.nmodes;
    hd.max_rank = (uint32_t)g.max_rank;
    hd.n = (uint64_t)g.n();
    hd.n_g = (uint64_t)g.n_g();
    hd.R0 = (uint64_t)g.R(0);
    hd.R1 = (uint64_t)g.R(1);
    hd.n_codes = (uint32_t)g.num.size();
    if (g.rp[2].empty()) g.rp[2].assign(1, 0);
    hd.n_out = (uint64_t)g.n_out();
    hd.R2 = (uint64_t)(g.rec[2].size() / 2);
    auto secs = sections(g);
    static const uint8_t zeros[64] = {0};
    Sha256 sh;
    uint64_t total = 0;
    for (auto &s : secs) {
        if (s.bytes) sh.update(s.ptr, s.bytes);
        size_t p = pad64(s.bytes) - s.bytes;
        if (p) sh.update(zeros, p);
        total += pad64(s.bytes);
    }
    hd.payload_bytes = total;
    sh.final(hd.sha256);
    memcpy(g.sha, hd.sha256, 32);
    std::string tmp = path + ".partial";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return "cannot open " + tmp + " for writing";
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1;
    for (auto &s : secs) {
        if (!ok) break;
        if (s.bytes) ok = fwrite(s.ptr, 1, s.bytes, f) == s.bytes;
        size_t p = pad64(s.bytes) - s.bytes;
        if (ok && p) ok = fwrite(zeros, 1, p, f) == p;
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) { remove(tmp.c_str()); return "write failed for " + tmp; }
    if (rename(tmp.c_str(), path.c_str()) != 0) return "cannot rename to " + path;
    if (bytes) *bytes = (int64_t)(sizeof(hd) + total);
    return "";
}

int read_bundle(const std::string &path, HostGraph &g, std::string *err) {
    FILE *f = fopen(path.c_str(), "rb");
    if (!f) { *err = "cannot open " + path; return 2; }
    std::unique_ptr<FILE, int (*)(FILE *)> guard(f, fclose);
    FileHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1) { *err = "truncated header"; return 3; }
    if (memcmp(hd.magic, kMagic, 8) != 0) { *err = "not a CUT graph bundle (bad magic)"; return 3; }
    if (hd.version != kVersion) { *err = "unsupported bundle version"; return 3; }
    if (hd.n == 0 || hd.n > kIndexMask || hd.n_g > kIndexMask || hd.n_codes == 0 ||
        hd.n_codes > (uint32_t)kMaxCodes || hd.nmodes == 0 || hd.nmodes > 32 || hd.algebra > 2) {
        *err = "bundle header out of range"; return 3;
    }
    g.algebra = (int)hd.algebra; g.nmodes = (int)hd.nmodes; g.max_rank = (int)hd.max_rank;
    try {
        g.labels.resize(hd.n); g.gen_labels.resize(hd.n_g); g.diag.resize(hd.n);
        g.num.resize(hd.n_codes); g.den.resize(hd.n_codes);
        g.rp[0].resize(hd.n_g + 1); g.rec[0].resize(2 * hd.R0);
        g.rp[1].resize(hd.n + 1); g.rec[1].resize(2 * hd.R1);
        g.out_labels.resize(hd.n_out); g.rp[2].resize(hd.n_out + 1); g.rec[2].resize(2 * hd.R2);
    } catch (...) { *err = "out of host memory reading bundle"; return 5; }
    auto secs = sections(g);
    uint64_t expect = 0;
    for (auto &s : secs) expect += pad64(s.bytes);
    if (expect != hd.payload_bytes) { *err = "payload size inconsistent with header"; return 3; }
    Sha256 sh;
    uint8_t padbuf[64];
    for (auto &s : secs) {
        if (s.bytes && fread(s.ptr, 1, s.bytes, f) != s.bytes) { *err = "truncated payload"; return 3; }
        if (s.bytes) sh.update(s.ptr, s.bytes);
        size_t p = pad64(s.bytes) - s.bytes;
        if (p) {
            if (fread(padbuf, 1, p, f) != p) { *err = "truncated payload"; return 3; }
            sh.update(padbuf, p);
        }
    }
    uint8_t dg[32];
    sh.final(dg);
    if (memcmp(dg, hd.sha256, 32) != 0) { *err = "payload SHA-256 mismatch"; return 4; }
    memcpy(g.sha, dg, 32);
    // structural validation
    if (hd.n_out > kIndexMask) { *err = "outside-space index beyond 2^24"; return 3; }
    for (int s = 0; s < 3; s++) {
        const auto &rp = g.rp[s];
        uint64_t rows = rp.size() - 1;
        uint64_t lim1 = s == 0 ? hd.n : hd.n_g;
        if (rp[0] != 0 || rp[rows] != g.rec[s].size() / 2) { *err = "row pointers do not span records"; return 3; }
        for (uint64_t r = 0; r < rows; r++)
            if (rp[r + 1] < rp[r]) { *err = "row pointers not monotone"; return 3; }
        const uint32_t *rc = g.rec[s].data();
        for (uint64_t e = 0; e < g.rec[s].size() / 2; e++) {
            uint32_t w0 = rc[2 * e], w1 = rc[2 * e + 1];
            if ((w0 & kIndexMask) >= lim1 || w1 >= hd.n || (w0 >> kIndexBits) >= hd.n_codes) {
                *err = "record index out of range"; return 3;
            }
        }
    }
    for (uint32_t c = 0; c < hd.n_codes; c++)
        if (g.den[c] <= 0) { *err = "non-positive factor denominator"; return 3; }
    return 0;
}

}  // namespace cut
