// checkpoint.cpp -- the checkpoint file of a resumable chunked sum and the
// chunk loop (checkpoint.h).
#include "checkpoint.h"

#include <errno.h>
#include <fcntl.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>

#include "zxp.h"

namespace zxp {
namespace ckpt {

namespace {

const char kMagic[8] = {'Z', 'X', 'P', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

template <class T>
void put(std::vector<uint8_t>& b, T v) {
    const size_t o = b.size();
    b.resize(o + sizeof v);
    memcpy(b.data() + o, &v, sizeof v);
}

template <class T>
bool get(const std::vector<uint8_t>& b, size_t& o, T* v) {
    if (o + sizeof *v > b.size()) return false;
    memcpy(v, b.data() + o, sizeof *v);
    o += sizeof *v;
    return true;
}

std::vector<uint8_t> encode(const State& st) {
    std::vector<uint8_t> b(kMagic, kMagic + 8);
    put(b, kVersion);
    put(b, st.width);
    put(b, st.digest);
    put(b, st.k);
    put(b, st.chunk_log2);
    put(b, st.n_chunks);
    put(b, st.e0);
    put(b, (uint32_t)0);
    for (int i = 0; i < 8; i++) put(b, st.sum[i]);
    put(b, st.done_count);
    b.insert(b.end(), st.done.begin(), st.done.end());
    put(b, fnv1a(b.data(), b.size()));
    return b;
}

bool write_all(int fd, const uint8_t* p, size_t n) {
    while (n) {
        const ssize_t w = ::write(fd, p, n);
        if (w < 0 && errno == EINTR) continue;
        if (w <= 0) return false;
        p += w;
        n -= (size_t)w;
    }
    return true;
}

uint64_t popcount_bytes(const std::vector<uint8_t>& v) {
    uint64_t c = 0;
    for (uint8_t x : v) c += (uint64_t)__builtin_popcount(x);
    return c;
}

}  // namespace

uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

State fresh(uint32_t width, uint64_t digest, uint32_t k, uint32_t chunk_log2, int32_t e0) {
    State st;
    st.width = width;
    st.digest = digest;
    st.k = k;
    st.chunk_log2 = chunk_log2 > k ? k : chunk_log2;
    st.n_chunks = ((1ull << k) + (1ull << st.chunk_log2) - 1) >> st.chunk_log2;
    st.e0 = e0;
    st.done.assign((size_t)((st.n_chunks + 7) / 8), 0);
    return st;
}

int load(const std::string& path, State* st) {
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return errno == ENOENT ? 0 : ZXP_EINVAL;
    std::vector<uint8_t> b;
    uint8_t buf[65536];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) b.insert(b.end(), buf, buf + r);
    const bool err = ferror(f) != 0;
    fclose(f);
    if (err || b.size() < 8 + sizeof(uint64_t) || memcmp(b.data(), kMagic, 8) != 0) return ZXP_EINVAL;
    uint64_t check = 0;
    memcpy(&check, b.data() + b.size() - sizeof check, sizeof check);
    if (fnv1a(b.data(), b.size() - sizeof check) != check) return ZXP_EINVAL;
    size_t o = 8;
    uint32_t version = 0, pad = 0;
    State s;
    if (!get(b, o, &version) || version != kVersion || !get(b, o, &s.width) || !get(b, o, &s.digest) ||
        !get(b, o, &s.k) || !get(b, o, &s.chunk_log2) || !get(b, o, &s.n_chunks) || !get(b, o, &s.e0) ||
        !get(b, o, &pad))
        return ZXP_EINVAL;
    for (int i = 0; i < 8; i++)
        if (!get(b, o, &s.sum[i])) return ZXP_EINVAL;
    if (!get(b, o, &s.done_count)) return ZXP_EINVAL;
    if ((s.width != 64 && s.width != 128) || s.k > 63 || s.chunk_log2 > s.k ||
        s.n_chunks != (((1ull << s.k) + (1ull << s.chunk_log2) - 1) >> s.chunk_log2))
        return ZXP_EINVAL;
    const size_t nb = (size_t)((s.n_chunks + 7) / 8);
    if (b.size() - sizeof check - o != nb) return ZXP_EINVAL;
    s.done.assign(b.begin() + (long)o, b.begin() + (long)(o + nb));
    if (popcount_bytes(s.done) != s.done_count) return ZXP_EINVAL;
    if (s.n_chunks % 8 && (s.done.back() >> (s.n_chunks % 8))) return ZXP_EINVAL;
    *st = std::move(s);
    return 1;
}

int save(const std::string& path, const State& st) {
    const std::vector<uint8_t> b = encode(st);
    const std::string tmp = path + ".tmp";
    const int fd = ::open(tmp.c_str(), O_WRONLY | O_CREAT | O_TRUNC, 0644);
    if (fd < 0) return ZXP_EINVAL;
    const bool ok = write_all(fd, b.data(), b.size()) && ::fsync(fd) == 0;
    if (::close(fd) != 0 || !ok || ::rename(tmp.c_str(), path.c_str()) != 0) {
        ::unlink(tmp.c_str());
        return ZXP_EINVAL;
    }
    // the rename itself reaches the disk with the directory
    const size_t slash = path.rfind('/');
    const std::string dir = slash == std::string::npos ? "." : (slash == 0 ? "/" : path.substr(0, slash));
    const int dfd = ::open(dir.c_str(), O_RDONLY);
    if (dfd >= 0) {
        ::fsync(dfd);
        ::close(dfd);
    }
    return ZXP_OK;
}

int run(const std::string& path, uint32_t width, uint64_t digest, uint32_t k, uint32_t chunk_log2, int32_t e0,
        uint64_t max_chunks, const ChunkFn& eval, State* out) {
    if ((width != 64 && width != 128) || k > 63) return ZXP_EINVAL;
    State st = fresh(width, digest, k, chunk_log2, e0);
    State old;
    const int ld = load(path, &old);
    if (ld < 0) return ld;
    if (ld == 1) {
        if (old.width != st.width || old.digest != st.digest || old.k != st.k ||
            old.chunk_log2 != st.chunk_log2 || old.e0 != st.e0)
            return ZXP_EINVAL;
        st = std::move(old);
    }
    const uint64_t total = 1ull << k, span = 1ull << st.chunk_log2;
    uint64_t ran = 0;
    for (uint64_t c = 0; c < st.n_chunks; c++) {
        if ((st.done[(size_t)(c >> 3)] >> (c & 7)) & 1) continue;
        if (max_chunks && ran == max_chunks) {
            *out = std::move(st);
            return ZXP_EAGAIN;
        }
        const uint64_t first = c << st.chunk_log2;
        const uint64_t count = total - first < span ? total - first : span;
        uint64_t lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
        const int r = eval(first, count, lo, hi);
        if (r != ZXP_OK) {
            *out = std::move(st);
            return r;
        }
        for (int i = 0; i < 4; i++) {
            if (width == 128) {
                const uint64_t l = st.sum[i] + lo[i];
                st.sum[4 + i] += hi[i] + (l < lo[i] ? 1u : 0u);
                st.sum[i] = l;
            } else {
                st.sum[i] += lo[i];
            }
        }
        st.done[(size_t)(c >> 3)] |= (uint8_t)(1u << (c & 7));
        st.done_count++;
        ran++;
        const int w = save(path, st);
        if (w != ZXP_OK) {
            *out = std::move(st);
            return w;
        }
    }
    // (every chunk run was saved; a state that was complete is left as it is)
    *out = std::move(st);
    return ZXP_OK;
}

}  // namespace ckpt
}  // namespace zxp
