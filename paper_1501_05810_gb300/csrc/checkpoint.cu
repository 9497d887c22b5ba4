// checkpoint.cu -- save and restore the state a time step reads.
//
// A checkpoint holds the body state exactly as the device keeps it (FP64
// positions with radii, quaternions, the velocity records with 1/m and 1/I
// in the sweep precision, the finite-mass flags), the parameters, the shared
// walls, the largest radius, the previous step's contacts with their
// world-frame impulses (what the warm start of the next step matches by
// key) and the warm-start network if one is loaded.  Restoring it into a
// scene with the same bodies, box and precision makes the next steps
// bit-identical to those of the scene that wrote it.
//
// File layout (host byte order): CkptHeader, then pos_r (n x 32 B), quat
// (n x 32 B), vel (2n x 16 B FP32 / 32 B FP64), finite (n B), then, if
// has_prev: row offsets by j1 (n + 1 u32), j2 (prev_count u32), world
// impulses (prev_count x 32 B), then, if has_mlp: 9,347 FP32 parameters.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "nbgs_internal.cuh"

namespace nbgs {

namespace {

constexpr char kMagic[8] = {'N', 'B', 'G', 'S', 'C', 'K', 'P', '1'};
constexpr uint32_t kVersion = 3;
constexpr int64_t kMlpParams = 9347;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n;
    int32_t fp32;
    int32_t has_prev;
    int64_t prev_count;
    int32_t has_mlp;
    int32_t reserved;
    double r_max;
    nbgs_params prm;
    Planes planes;
};

struct File {
    FILE* f = nullptr;
    ~File()
    {
        if (f) fclose(f);
    }
};

bool put(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool get(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

template <class T>
nbgs_status d2h(nbgs_scene* s, std::vector<T>& h, const void* d, size_t count)
{
    h.resize(count);
    if (count == 0) return NBGS_OK;
    return cuda_check(s, cudaMemcpyAsync(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost, s->stream),
                      "save_state: copy");
}

}  // namespace

nbgs_status run_save_state(nbgs_scene* s, const char* path)
{
    if (!path) return fail(s, NBGS_EINVAL, "save_state: null path");
    if (s->batch || s->composite) return fail(s, NBGS_EINVAL, "save_state: batched and composite scenes are not supported");
    const int64_t n = s->n;
    const size_t vbytes = s->fp32 ? 16 : 32;
    // the contacts the next step's warm start reads: the last solved step's
    // (still in the current arrays), or those of a checkpoint not yet stepped
    const bool warm = s->prm.warm_start != NBGS_WARM_NONE;
    const bool cur = warm && s->solved;
    const bool kept = warm && !cur && s->have_prev;
    CkptHeader h{};
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.version = kVersion;
    h.header_bytes = sizeof(CkptHeader);
    h.n = n;
    h.fp32 = s->fp32 ? 1 : 0;
    h.has_prev = (cur || kept) ? 1 : 0;
    h.prev_count = cur ? s->n_contacts : (kept ? s->prev_count : 0);
    h.has_mlp = s->mlp_theta ? 1 : 0;
    h.r_max = s->r_max;
    h.prm = s->prm;
    h.planes = s->planes;

    std::vector<unsigned char> pos, quat, vel, fin;
    std::vector<uint32_t> off, j2;
    std::vector<unsigned char> P;
    std::vector<float> theta;
    nbgs_status rc = d2h(s, pos, s->pos_r, (size_t)n * 32);
    if (rc == NBGS_OK) rc = d2h(s, quat, s->quat, (size_t)n * 32);
    if (rc == NBGS_OK) rc = d2h(s, vel, s->vel, (size_t)n * 2 * vbytes);
    if (rc == NBGS_OK) rc = d2h(s, fin, s->finite, (size_t)n);
    if (rc == NBGS_OK && h.has_prev) {
        rc = d2h(s, off, cur ? s->row_off : s->prev_row_off, (size_t)n + 1);
        if (rc == NBGS_OK) rc = d2h(s, j2, cur ? s->cj2 : s->prev_j2, (size_t)h.prev_count);
        const void* pw = cur ? (const void*)s->cworld : (const void*)s->prev_P;
        if (rc == NBGS_OK) rc = d2h(s, P, pw, (size_t)h.prev_count * 32);
    }
    if (rc == NBGS_OK && h.has_mlp) rc = d2h(s, theta, s->mlp_theta, (size_t)kMlpParams);
    if (rc == NBGS_OK) rc = cuda_check(s, cudaStreamSynchronize(s->stream), "save_state");
    if (rc != NBGS_OK) return rc;

    File f;
    f.f = fopen(path, "wb");
    if (!f.f) return fail(s, NBGS_EINVAL, std::string("save_state: cannot open ") + path);
    bool ok = put(f.f, &h, sizeof(h)) && put(f.f, pos.data(), pos.size()) && put(f.f, quat.data(), quat.size()) &&
              put(f.f, vel.data(), vel.size()) && put(f.f, fin.data(), fin.size());
    if (ok && h.has_prev)
        ok = put(f.f, off.data(), off.size() * 4) && put(f.f, j2.data(), j2.size() * 4) && put(f.f, P.data(), P.size());
    if (ok && h.has_mlp) ok = put(f.f, theta.data(), theta.size() * 4);
    if (ok) ok = fflush(f.f) == 0;
    if (!ok) return fail(s, NBGS_EINVAL, std::string("save_state: write failed: ") + path);
    return NBGS_OK;
}

nbgs_status grow_contacts(nbgs_scene* s, int64_t need);  // api.cu
bool params_valid(const nbgs_params* p);                  // api.cu

nbgs_status run_load_state(nbgs_scene* s, const char* path)
{
    if (!path) return fail(s, NBGS_EINVAL, "load_state: null path");
    if (s->batch || s->composite) return fail(s, NBGS_EINVAL, "load_state: batched and composite scenes are not supported");
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return fail(s, NBGS_EINVAL, std::string("load_state: cannot open ") + path);
    CkptHeader h{};
    if (!get(f.f, &h, sizeof(h)) || std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != kVersion ||
        h.header_bytes != sizeof(CkptHeader))
        return fail(s, NBGS_EINVAL, "load_state: not a checkpoint of this library version");
    if (h.n != s->n || (h.fp32 != 0) != s->fp32)
        return fail(s, NBGS_EINVAL, "load_state: the scene has another body count or sweep precision");
    for (int a = 0; a < 3; ++a)
        if (h.prm.box_lo[a] != s->prm.box_lo[a] || h.prm.box_hi[a] != s->prm.box_hi[a] ||
            (h.prm.periodic[a] != 0) != (s->prm.periodic[a] != 0))
            return fail(s, NBGS_EINVAL, "load_state: the scene has another box");
    // everything below indexes device arrays or sizes the cell grid: the
    // header must hold what a scene of this library can hold
    if (h.planes.count < 0 || h.planes.count > kMaxPlanes || h.planes.ncones < 0 || h.planes.ncones > kMaxCones ||
        h.prev_count < 0 || h.prev_count > 0xFFFFFFF0LL || (h.has_prev && h.prm.warm_start == NBGS_WARM_NONE) ||
        !params_valid(&h.prm) || (h.prm.precision == NBGS_FP32) != s->fp32 || !std::isfinite(h.r_max) ||
        !(h.r_max >= 0.0))
        return fail(s, NBGS_EINVAL, "load_state: corrupt header");
    const int64_t n = s->n;
    const size_t vbytes = s->fp32 ? 16 : 32;
    std::vector<unsigned char> pos((size_t)n * 32), quat((size_t)n * 32), vel((size_t)n * 2 * vbytes), fin((size_t)n);
    std::vector<uint32_t> off, j2;
    std::vector<unsigned char> P;
    std::vector<float> theta;
    bool ok = get(f.f, pos.data(), pos.size()) && get(f.f, quat.data(), quat.size()) &&
              get(f.f, vel.data(), vel.size()) && get(f.f, fin.data(), fin.size());
    if (ok && h.has_prev) {
        off.resize((size_t)n + 1);
        j2.resize((size_t)h.prev_count);
        P.resize((size_t)h.prev_count * 32);
        ok = get(f.f, off.data(), off.size() * 4) && get(f.f, j2.data(), j2.size() * 4) && get(f.f, P.data(), P.size());
        if (ok) ok = off[0] == 0 && (int64_t)off[n] == h.prev_count;
        for (int64_t i = 0; ok && i < n; ++i) ok = off[i] <= off[i + 1];   // rows inside [0, prev_count]
    }
    // radii (the fourth word of every position record) within the largest
    // radius the cell grid is sized for
    for (int64_t i = 0; ok && i < n; ++i) {
        double r;
        std::memcpy(&r, &pos[(size_t)i * 32 + 24], sizeof(r));
        ok = r >= 0.0 && r <= h.r_max;
    }
    if (ok && h.has_mlp) {
        theta.resize((size_t)kMlpParams);
        ok = get(f.f, theta.data(), theta.size() * 4);
    }
    if (!ok) return fail(s, NBGS_EINVAL, "load_state: truncated or inconsistent file");

    // the warm-start arrays must hold prev_count contacts
    s->have_prev = false;
    if (h.prev_count > s->ccap) {
        nbgs_status rc = grow_contacts(s, h.prev_count);
        if (rc != NBGS_OK) return rc;
    }
    if (h.has_mlp && !s->mlp_theta) {
        s->mlp_theta = (float*)dev_alloc(s, (size_t)kMlpParams * sizeof(float));
        if (!s->mlp_theta) return fail(s, NBGS_ENOMEM, "load_state: allocation");
    }
    cudaStream_t st = s->stream;
    cudaMemcpyAsync(s->pos_r, pos.data(), pos.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->quat, quat.data(), quat.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->vel, vel.data(), vel.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s->finite, fin.data(), fin.size(), cudaMemcpyHostToDevice, st);
    if (h.has_prev) {
        cudaMemcpyAsync(s->prev_row_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice, st);
        if (h.prev_count > 0) {
            cudaMemcpyAsync(s->prev_j2, j2.data(), j2.size() * 4, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(s->prev_P, P.data(), P.size(), cudaMemcpyHostToDevice, st);
        }
    }
    if (h.has_mlp) cudaMemcpyAsync(s->mlp_theta, theta.data(), theta.size() * 4, cudaMemcpyHostToDevice, st);
    nbgs_status rc = cuda_check(s, cudaStreamSynchronize(st), "load_state");   // the host buffers go out of scope
    if (rc != NBGS_OK) return rc;
    s->prm = h.prm;
    s->planes = h.planes;
    s->r_max = h.r_max;
    s->detected = s->coloured = s->solved = false;
    s->n_contacts = 0;
    s->have_prev = h.has_prev != 0;
    s->prev_count = h.has_prev ? h.prev_count : 0;
    return NBGS_OK;
}

}  // namespace nbgs

extern "C" {

nbgs_status nbgs_save_state(nbgs_scene* s, const char* path)
{
    if (!s) return NBGS_EINVAL;
    if (s->status != NBGS_OK) return s->status;
    return nbgs::run_save_state(s, path);
}

nbgs_status nbgs_load_state(nbgs_scene* s, const char* path)
{
    if (!s) return NBGS_EINVAL;
    if (s->status != NBGS_OK) return s->status;
    return nbgs::run_load_state(s, path);
}

}  // extern "C"
