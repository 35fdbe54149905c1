// kl_config.cpp -- configuration space, wisdom files, selection heuristic,
// grid validation and vertical profiles (host code only).
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>

#include "kl_internal.h"

namespace kl {

// ============================================================ config text

static const char *kPermNames[6] = {"XYZ", "XZY", "YXZ", "YZX", "ZXY", "ZYX"};

std::string config_string(const Config &c)
{
    char b[512];
    if (c.family == 0) {
        snprintf(b, sizeof b,
                 "direct:bx=%d,by=%d,bz=%d,tx=%d,ty=%d,tz=%d,ux=%d,uy=%d,uz=%d,"
                 "cx=%d,cy=%d,cz=%d,perm=%s,minb=%d",
                 c.bx, c.by, c.bz, c.tx, c.ty, c.tz, c.ux, c.uy, c.uz, c.cx, c.cy, c.cz,
                 kPermNames[c.perm], c.minb);
    } else if (c.family == 1) {
        snprintf(b, sizeof b, "zmarch:bx=%d,by=%d,px=%d,py=%d,kc=%d,ns=%d,minb=%d", c.mbx, c.mby,
                 c.mpx, c.mpy, c.kc, c.ns, c.mminb);
    } else {
        snprintf(b, sizeof b, "zpack:w=%d,ly=%d,kc=%d,ns=%d,minb=%d,yx=%d,pk=%d,cs=%d%s", c.mby,
                 c.mpy, c.kc, c.ns, c.mminb, c.yx, c.pk, c.cs,
                 c.pe == 1 ? ",pe=1" : c.pe == 2 ? ",pe=2" : "");
    }
    return b;
}

static bool parse_int(const std::string &v, int *out)
{
    char *end = nullptr;
    errno = 0;
    long x = strtol(v.c_str(), &end, 10);
    if (errno || end == v.c_str() || *end) return false;
    *out = (int)x;
    return true;
}

bool config_parse(const std::string &text, Config *c, std::string *err)
{
    std::string s = text;
    while (!s.empty() && isspace((unsigned char)s.back())) s.pop_back();
    while (!s.empty() && isspace((unsigned char)s.front())) s.erase(s.begin());
    *c = Config();
    if (s.empty() || s == "default" || s == "direct" || s == "direct:default") return true;
    std::string body;
    size_t colon = s.find(':');
    std::string fam = colon == std::string::npos ? s : s.substr(0, colon);
    body = colon == std::string::npos ? "" : s.substr(colon + 1);
    if (fam == "direct") c->family = 0;
    else if (fam == "zmarch") c->family = 1;
    else if (fam == "zpack") {
        c->family = 2;
        c->mbx = 32;
        c->mpx = 2;
        c->mby = 8;
        c->mpy = 2;
    } else {
        *err = "unknown configuration family '" + fam + "'";
        return false;
    }
    std::stringstream ss(body);
    std::string item;
    while (std::getline(ss, item, ',')) {
        if (item.empty()) continue;
        size_t eq = item.find('=');
        if (eq == std::string::npos) {
            *err = "configuration item without '=': " + item;
            return false;
        }
        std::string k = item.substr(0, eq), v = item.substr(eq + 1);
        int x = 0;
        if (k == "perm" && c->family == 0) {
            int p = -1;
            for (int q = 0; q < 6; ++q)
                if (v == kPermNames[q]) p = q;
            if (p < 0 && !(parse_int(v, &p) && p >= 0 && p < 6)) {
                *err = "bad unravel permutation '" + v + "'";
                return false;
            }
            c->perm = p;
            continue;
        }
        if (!parse_int(v, &x)) {
            *err = "bad integer for '" + k + "': " + v;
            return false;
        }
        int *dst = nullptr;
        if (c->family == 0) {
            if (k == "bx") dst = &c->bx; else if (k == "by") dst = &c->by; else if (k == "bz") dst = &c->bz;
            else if (k == "tx") dst = &c->tx; else if (k == "ty") dst = &c->ty; else if (k == "tz") dst = &c->tz;
            else if (k == "ux") dst = &c->ux; else if (k == "uy") dst = &c->uy; else if (k == "uz") dst = &c->uz;
            else if (k == "cx") dst = &c->cx; else if (k == "cy") dst = &c->cy; else if (k == "cz") dst = &c->cz;
            else if (k == "minb") dst = &c->minb;
        } else if (c->family == 2) {
            if (k == "w") dst = &c->mby; else if (k == "ly") dst = &c->mpy;
            else if (k == "yx") dst = &c->yx;
            else if (k == "pk") dst = &c->pk;
            else if (k == "cs") dst = &c->cs;
            else if (k == "pe") dst = &c->pe;
            else if (k == "kc") dst = &c->kc; else if (k == "ns") dst = &c->ns;
            else if (k == "minb") dst = &c->mminb;
        } else {
            if (k == "bx") dst = &c->mbx; else if (k == "by") dst = &c->mby;
            else if (k == "px") dst = &c->mpx; else if (k == "py") dst = &c->mpy;
            else if (k == "kc") dst = &c->kc; else if (k == "ns") dst = &c->ns;
            else if (k == "minb") dst = &c->mminb;
        }
        if (!dst) {
            *err = "unknown configuration key '" + k + "'";
            return false;
        }
        *dst = x;
    }
    return true;
}

int esize_of(int dtype) { return dtype == KL_F64 ? 8 : dtype == KL_F32 ? 4 : 2; }
int halo_of(const kl_op &op) { return op.adv == 5 ? 3 : 1; }

static int round_up(int a, int b) { return (a + b - 1) / b * b; }

// zmarch shared-memory plane: rows of (L + TXS + R) elements, TYS + 2H rows;
// identical formulas to the KL_PITCH / KL_ROWS / KL_PLANE_BYTES macros of
// kl_stencil.cuh
ZGeom zmarch_geometry(const kl_op &op, const Config &c)
{
    ZGeom z;
    int es = esize_of(op.dtype), h = halo_of(op);
    z.al = 16 / es;
    z.txs = c.mbx * c.mpx;
    z.tys = c.mby * c.mpy;
    z.lpad = round_up(h, z.al);
    z.pitch = round_up(z.lpad + z.txs + h, z.al);
    z.rows = z.tys + 2 * h;
    z.halo = h;
    z.box_bytes = (size_t)z.pitch * z.rows * es;
    z.plane_bytes = (z.box_bytes + 127) / 128 * 128;
    z.nf = op.diff == 2 ? 4 : 3;
    return z;
}

size_t zmarch_smem_bytes(const kl_op &op, const Config &c)
{
    ZGeom z = zmarch_geometry(op, c);
    // ring + 128 B of alignment slack + one 8-byte mbarrier per slot
    size_t bytes = z.plane_bytes * z.nf * c.ns + 256;
    if (c.family == 2 && op.diff == 2) {
        // zpack, variable nu: u, v, w ring + a nu ring of tys + 2 rows per
        // plane, ns - 2R + 2 planes (ns - R + 1 for a carried ring of fewer
        // than 2R + 2 slots); no x-wrap strips
        size_t nplane = ((size_t)z.pitch * (z.tys + 2) * esize_of(op.dtype) + 127) / 128 * 128;
        const int nns = c.ns < 2 * z.halo + 2 ? c.ns - z.halo + 1 : c.ns - 2 * z.halo + 2;
        bytes = z.plane_bytes * 3 * c.ns + nplane * nns + 256;
    } else if (c.family == 2) {
        // zpack x-wrap strips: 3 fields x rows x 32 bytes per slot (128-B multiples)
        bytes += 3 * (size_t)((z.rows * 32 + 127) / 128 * 128) * c.ns;
    }
    // zpack y-face exchange: 3 fields x warps x 32 lanes x one packed pair;
    // one level ahead (yx=2) by level parity, with the tile's top faces and
    // its scalar x side faces
    const size_t pair = op.dtype == KL_F64 ? 16 : 8, scal = op.dtype == KL_F64 ? 8 : 4;
    if (c.family == 2 && c.yx == 1) bytes += 3 * (size_t)c.mby * 32 * pair + 16;
    if (c.family == 2 && c.yx == 2)
        bytes += 2 * 3 * ((size_t)c.mby * 32 * pair + 32 * pair + (size_t)z.tys * scal) + 16;
    return bytes;
}

static bool in(int v, std::initializer_list<int> set)
{
    for (int s : set)
        if (v == s) return true;
    return false;
}

bool config_check(const kl_op &op, const Config &c, std::string *err)
{
    if (c.family == 0) {
        if (!in(c.bx, {16, 32, 64, 128, 256}) || !in(c.by, {1, 2, 4, 8, 16}) ||
            !in(c.bz, {1, 2, 4, 8, 16})) {
            *err = "block size outside the space (bx 16..256, by/bz 1..16, powers of 2)";
            return false;
        }
        if (!in(c.tx, {1, 2, 4}) || !in(c.ty, {1, 2, 4}) || !in(c.tz, {1, 2, 4})) {
            *err = "tile factor outside {1,2,4}";
            return false;
        }
        for (int b : {c.ux, c.uy, c.uz, c.cx, c.cy, c.cz})
            if (b != 0 && b != 1) {
                *err = "unroll/contiguous flags must be 0 or 1";
                return false;
            }
        if (c.perm < 0 || c.perm > 5 || c.minb < 1 || c.minb > 6) {
            *err = "perm must be 0..5 and minb 1..6";
            return false;
        }
        if (c.bx * c.by * c.bz > 1024) {
            *err = "more than 1024 threads per block";
            return false;
        }
        return true;
    }
    if (c.family == 1 || c.family == 2) {
        if (c.family == 1 &&
            (!in(c.mbx, {32, 64, 128}) || !in(c.mby, {1, 2, 4, 8, 16}) || !in(c.mpx, {1, 2, 4}) ||
             !in(c.mpy, {1, 2, 4}))) {
            *err = "zmarch parameter outside the space";
            return false;
        }
        if (c.family == 2 && (c.mbx != 32 || c.mpx != 2 || !in(c.mby, {1, 2, 3, 4, 6, 7, 8, 9, 12, 16}) ||
                              !in(c.mpy, {1, 2, 3, 4, 5, 6, 8}))) {
            *err = "zpack parameter outside the space (w 1..16, ly 1..8)";
            return false;
        }
        if (c.family == 2 &&
            ((c.yx < 0 || c.yx > 2) || (c.pk != 0 && c.pk != 1) || (c.cs != 0 && c.cs != 1) ||
             (c.pe < 0 || c.pe > 2))) {
            *err = "yx and pe must be 0..2, pk and cs 0 or 1";
            return false;
        }
        if (c.family == 2 && c.cs && c.yx) {
            *err = "cs=1 forms every y face in its own warp group (yx must be 0)";
            return false;
        }
        if (c.family == 2 && op.diff == 2 && (c.cs || c.yx)) {
            *err = "zpack with variable nu needs cs=0 and yx=0";
            return false;
        }
        if (!in(c.kc, {4, 8, 16, 32, 64, 128, 256}) ||
            !(in(c.ns, {8, 9, 10, 12}) || (c.family == 2 && in(c.ns, {6, 7}))) ||
            c.mminb < 1 || c.mminb > 4) {
            *err = "z-march parameter outside the space";
            return false;
        }
        if (c.mbx * zmarch_block_y(c) > 1024) {
            *err = "more than 1024 threads per block";
            return false;
        }
        if (c.mminb * c.mbx * zmarch_block_y(c) > 2048) {
            *err = "minb x threads per block exceeds 2048 threads per SM";
            return false;
        }
        int reach = halo_of(op);
        // zpack (one warp group) may carry plane k-2 in registers (ring of
        // planes k-1 .. k+R plus one in flight: 2R slots)
        const bool carry_ok = c.family == 2 && !c.cs && reach >= 2;
        if (c.family == 2 && c.yx == 2 && !(carry_ok && op.diff != 2 && c.ns < 2 * reach + 2)) {
            *err = "yx=2 needs a ring of fewer than 2R+2 slots (2R or 2R+1), constant nu and cs=0";
            return false;
        }
        if (c.ns < 2 * reach + 2 && !(carry_ok && c.ns >= 2 * reach)) {
            *err = carry_ok ? "plane ring needs at least 2R slots"
                            : "plane ring needs at least 2R+2 slots";
            return false;
        }
        ZGeom z = zmarch_geometry(op, c);
        if (z.pitch > 256 || z.rows > 256) {
            *err = "TMA box wider than 256 elements";
            return false;
        }
        size_t smem = zmarch_smem_bytes(op, c);
        if ((size_t)c.mminb * smem > 228u * 1024u || smem > 227u * 1024u) {
            *err = "shared memory " + std::to_string(smem) + " B x minb exceeds the SM";
            return false;
        }
        return true;
    }
    *err = "unknown family";
    return false;
}

// Raw (unconstrained) spaces.  direct = Table 2: 5*5*5 block shapes x 3^3 tile
// factors x 2^3 unroll x 2^3 contiguous x 6 permutations x 6 min-blocks.
static const int kBX[] = {16, 32, 64, 128, 256}, kBYZ[] = {1, 2, 4, 8, 16}, kT[] = {1, 2, 4};
static const int kMBX[] = {32, 64, 128}, kMBY[] = {1, 2, 4, 8, 16}, kMP[] = {1, 2, 4},
                 kKC[] = {4, 8, 16, 32, 64, 128, 256}, kNS[] = {8, 9, 10, 12};

static const int kW[] = {1, 2, 3, 4, 6, 7, 8, 9, 12, 16}, kLY[] = {1, 2, 3, 4, 5, 6, 8}, kNSP[] = {6, 7, 8, 9, 10, 12};

int64_t space_size(int family)
{
    if (family == 0) return 5LL * 5 * 5 * 27 * 8 * 8 * 6 * 6;
    if (family == 1) return 3LL * 5 * 3 * 3 * 7 * 4 * 4;
    if (family == 2) return 10LL * 7 * 7 * 6 * 4 * 3 * 2 * 3;
    return 0;
}

bool space_config(int family, int64_t idx, Config *c)
{
    if (idx < 0 || idx >= space_size(family)) return false;
    *c = Config();
    c->family = family;
    auto take = [&](int radix) {
        int r = (int)(idx % radix);
        idx /= radix;
        return r;
    };
    if (family == 0) {
        c->bx = kBX[take(5)];
        c->by = kBYZ[take(5)];
        c->bz = kBYZ[take(5)];
        c->tx = kT[take(3)];
        c->ty = kT[take(3)];
        c->tz = kT[take(3)];
        c->ux = take(2); c->uy = take(2); c->uz = take(2);
        c->cx = take(2); c->cy = take(2); c->cz = take(2);
        c->perm = take(6);
        c->minb = 1 + take(6);
    } else if (family == 2) {
        c->mbx = 32;
        c->mpx = 2;
        c->mby = kW[take(10)];
        c->mpy = kLY[take(7)];
        c->kc = kKC[take(7)];
        c->ns = kNSP[take(6)];
        c->mminb = 1 + take(4);
        c->yx = take(3);
        c->cs = take(2);
        c->pe = take(3);
    } else {
        c->mbx = kMBX[take(3)];
        c->mby = kMBY[take(5)];
        c->mpx = kMP[take(3)];
        c->mpy = kMP[take(3)];
        c->kc = kKC[take(7)];
        c->ns = kNS[take(4)];
        c->mminb = 1 + take(4);
    }
    return true;
}

// =============================================================== wisdom

// key=value tokens; a value may be "double quoted" (no escapes inside)
static bool tokenize(const std::string &line, std::map<std::string, std::string> *kv,
                     std::string *err)
{
    size_t p = 0, n = line.size();
    while (p < n) {
        while (p < n && isspace((unsigned char)line[p])) ++p;
        if (p >= n) break;
        size_t eq = line.find('=', p);
        if (eq == std::string::npos) {
            *err = "token without '='";
            return false;
        }
        std::string key = line.substr(p, eq - p);
        if (key.empty() || key.find(' ') != std::string::npos) {
            *err = "bad key";
            return false;
        }
        p = eq + 1;
        std::string val;
        if (p < n && line[p] == '"') {
            size_t q = line.find('"', p + 1);
            if (q == std::string::npos) {
                *err = "unterminated quote";
                return false;
            }
            val = line.substr(p + 1, q - p - 1);
            p = q + 1;
        } else {
            size_t q = p;
            while (q < n && !isspace((unsigned char)line[q])) ++q;
            val = line.substr(p, q - p);
            p = q;
        }
        (*kv)[key] = val;
    }
    return true;
}

bool wisdom_read(const std::string &path, std::vector<WisdomRecord> *out, std::string *err)
{
    out->clear();
    std::ifstream in(path);
    if (!in) {
        *err = "cannot open wisdom file " + path;
        return false;
    }
    std::string line;
    int lineno = 0;
    while (std::getline(in, line)) {
        ++lineno;
        size_t s = line.find_first_not_of(" \t\r");
        if (s == std::string::npos || line[s] == '#') continue;
        std::map<std::string, std::string> kv;
        std::string e;
        if (!tokenize(line, &kv, &e)) {
            *err = path + ":" + std::to_string(lineno) + ": " + e;
            return false;
        }
        WisdomRecord r;
        auto need = [&](const char *k) -> const std::string * {
            auto it = kv.find(k);
            return it == kv.end() ? nullptr : &it->second;
        };
        const std::string *dev = need("device"), *cc = need("cc"), *nx = need("nx"),
                          *ny = need("ny"), *nz = need("nz"), *cfg = need("config");
        if (!dev || !cc || !nx || !ny || !nz || !cfg) {
            *err = path + ":" + std::to_string(lineno) + ": record lacks device/cc/nx/ny/nz/config";
            return false;
        }
        r.device = *dev;
        if (sscanf(cc->c_str(), "%d.%d", &r.cc_major, &r.cc_minor) != 2 ||
            !parse_int(*nx, &r.nx) || !parse_int(*ny, &r.ny) || !parse_int(*nz, &r.nz)) {
            *err = path + ":" + std::to_string(lineno) + ": bad cc or size";
            return false;
        }
        const std::string *zbc = need("zbc");
        if (zbc && !parse_int(*zbc, &r.zbc)) {
            *err = path + ":" + std::to_string(lineno) + ": bad zbc";
            return false;
        }
        r.config = *cfg;
        if (const std::string *t = need("time_us")) r.time_us = atof(t->c_str());
        for (auto &p : kv)
            if (p.first != "device" && p.first != "cc" && p.first != "nx" && p.first != "ny" &&
                p.first != "nz" && p.first != "config" && p.first != "zbc" && p.first != "time_us")
                r.extra[p.first] = p.second;
        out->push_back(r);
    }
    return true;
}

// Rules 2-5 of the Sec. 4.5 heuristic with a given distance between a
// record's size and the problem: the nearest record of this device, else of
// this compute capability, else of any device, else the default.  Records of
// one size (several tuning sessions) compete as in rule 1 (the fastest, ties
// to the newest); different sizes at the same distance go by file order.
// Records of another zbc are never chosen.
template <class Dist>
static int select_nearest(const std::vector<WisdomRecord> &recs, const std::string &device, int ccM,
                          int ccm, int zbc, Dist dist, std::string *config)
{
    auto nearest = [&](auto pred) -> const WisdomRecord * {
        const WisdomRecord *best = nullptr;
        double bd = 0;
        for (const WisdomRecord &r : recs) {
            if (r.zbc != zbc || !pred(r)) continue;
            double d = dist(r);
            const bool same_size = best && r.nx == best->nx && r.ny == best->ny && r.nz == best->nz;
            if (!best || d < bd || (same_size && r.time_us <= best->time_us)) {
                best = &r;
                bd = d;
            }
        }
        return best;
    };
    if (const WisdomRecord *r = nearest([&](const WisdomRecord &x) { return x.device == device; })) {
        *config = r->config;
        return 2;
    }
    if (const WisdomRecord *r = nearest([&](const WisdomRecord &x) {
            return x.cc_major == ccM && x.cc_minor == ccm;
        })) {
        *config = r->config;
        return 3;
    }
    if (const WisdomRecord *r = nearest([&](const WisdomRecord &) { return true; })) {
        *config = r->config;
        return 4;
    }
    *config = "default";
    return 5;
}

// Sec. 4.5 heuristic.  Rule 1: a record of this device and exactly this size
// (several: the fastest, ties to the newest); then the nearest size in
// Euclidean distance over (nx, ny, nz), by the tiers of select_nearest.
int wisdom_select(const std::vector<WisdomRecord> &recs, const std::string &device, int ccM,
                  int ccm, int zbc, int nx, int ny, int nz, std::string *config)
{
    const WisdomRecord *exact = nullptr;
    for (const WisdomRecord &r : recs)
        if (r.zbc == zbc && r.device == device && r.nx == nx && r.ny == ny && r.nz == nz)
            if (!exact || r.time_us <= exact->time_us) exact = &r;
    if (exact) {
        *config = exact->config;
        return 1;
    }
    return select_nearest(recs, device, ccM, ccm, zbc, [&](const WisdomRecord &r) {
        double a = r.nx - nx, b = r.ny - ny, c = r.nz - nz;
        return std::sqrt(a * a + b * b + c * c);
    }, config);
}

// A batch's configuration: the record whose tuned problem has the point count
// nearest (in ratio) to the batch's total, by the tiers of select_nearest.  A
// batch offers the parallelism of all its grids together, so the record
// tuned for a problem of that size fits it better than the small-grid
// records, tuned to spread one small grid over the device.
int wisdom_select_points(const std::vector<WisdomRecord> &recs, const std::string &device, int ccM,
                         int ccm, int zbc, double points, std::string *config)
{
    const double lp = std::log(std::max(points, 1.0));
    return select_nearest(recs, device, ccM, ccm, zbc, [&](const WisdomRecord &r) {
        const double v = std::max(1.0, (double)r.nx * r.ny * r.nz);
        return std::fabs(std::log(v) - lp);
    }, config);
}

static const char *dtype_name(int d)
{
    return d == KL_F64 ? "f64" : d == KL_F32 ? "f32" : d == KL_BF16 ? "bf16" : "f16";
}

std::string wisdom_file_name(const kl_op &op)
{
    char b[128];
    snprintf(b, sizeof b, "tendency_adv%d_diff%d_%s%s.wisdom", op.adv, op.diff,
             dtype_name(op.dtype), op.accumulate ? "_acc" : "");
    return b;
}

bool wisdom_append(const std::string &path, const WisdomRecord &r, std::string *err)
{
    bool exists = false;
    {
        std::ifstream t(path);
        exists = (bool)t;
    }
    FILE *f = fopen(path.c_str(), "a");
    if (!f) {
        *err = "cannot open wisdom file for append: " + path;
        return false;
    }
    if (!exists)
        fprintf(f, "# kl wisdom file: one record per tuning session (device x problem size)\n");
    fprintf(f, "device=\"%s\" cc=%d.%d zbc=%d nx=%d ny=%d nz=%d config=\"%s\" time_us=%.3f",
            r.device.c_str(), r.cc_major, r.cc_minor, r.zbc, r.nx, r.ny, r.nz, r.config.c_str(),
            r.time_us);
    for (auto &p : r.extra) {
        bool quote = p.second.find_first_of(" \t") != std::string::npos || p.second.empty();
        fprintf(f, quote ? " %s=\"%s\"" : " %s=%s", p.first.c_str(), p.second.c_str());
    }
    fprintf(f, "\n");
    bool ok = fclose(f) == 0;
    if (!ok) *err = "write failed: " + path;
    return ok;
}

// ============================================================ compile keys

std::string compile_defines(const kl_op &op, const Config &c, int zbc, int zuni)
{
    char b[512];
    int n = snprintf(b, sizeof b, "-DKL_DTYPE=%d -DKL_ADV=%d -DKL_DIFF=%d -DKL_ZBC=%d -DKL_ZUNI=%d "
                     "-DKL_ACC=%d -DKL_OF32=%d -DKL_FAMILY=%d", op.dtype, op.adv, op.diff, zbc, zuni,
                     op.accumulate ? 1 : 0, op.out_f32 ? 1 : 0, c.family);
    if (c.family == 0) {
        snprintf(b + n, sizeof b - n,
                 " -DKL_BX=%d -DKL_BY=%d -DKL_BZ=%d -DKL_TX=%d -DKL_TY=%d -DKL_TZ=%d -DKL_UX=%d"
                 " -DKL_UY=%d -DKL_UZ=%d -DKL_CX=%d -DKL_CY=%d -DKL_CZ=%d -DKL_PERM=%d -DKL_MINB=%d",
                 c.bx, c.by, c.bz, c.tx, c.ty, c.tz, c.ux, c.uy, c.uz, c.cx, c.cy, c.cz, c.perm,
                 c.minb);
    } else {
        snprintf(b + n, sizeof b - n,
                 " -DKL_MBX=%d -DKL_MBY=%d -DKL_MPX=%d -DKL_MPY=%d -DKL_KC=%d -DKL_NS=%d"
                 " -DKL_MMINB=%d -DKL_YX=%d -DKL_PK=%d -DKL_CS=%d -DKL_PE=%d",
                 c.mbx, c.mby, c.mpx, c.mpy, c.kc, c.ns, c.mminb, c.family == 2 ? c.yx : 0,
                 c.family == 2 ? c.pk : 1, c.family == 2 ? c.cs : 0, c.family == 2 ? c.pe : 0);
    }
    return b;
}

// ====================================================== grid validation

kl_status check_grid(const kl_grid *g, int need_g, Geom *geo)
{
    if (!g) return fail(KL_ERR_INVALID_ARG, "grid is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(KL_ERR_INVALID_ARG, "interior extents must be >= 1");
    if (g->g < need_g)
        return fail(KL_ERR_INVALID_ARG, "ghost width " + std::to_string(g->g) + " < required " +
                                            std::to_string(need_g));
    if (g->g > g->nx || g->g > g->ny || g->g >= g->nz + (g->zbc == 0 ? 1 : 0))
        return fail(KL_ERR_INVALID_ARG, "ghost width larger than the grid");
    if (g->zbc != 0 && g->zbc != 1) return fail(KL_ERR_INVALID_ARG, "zbc must be 0 or 1");
    if (g->xybc != 0 && g->xybc != 1) return fail(KL_ERR_INVALID_ARG, "xybc must be 0 or 1");
    if (!(g->dx > 0) || !(g->dy > 0)) return fail(KL_ERR_INVALID_ARG, "dx, dy must be > 0");
    if (!g->zh && !(g->dz > 0)) return fail(KL_ERR_INVALID_ARG, "dz must be > 0 when zh is NULL");
    if (g->zh)
        for (int k = 0; k < g->nz; ++k)
            if (!(g->zh[k + 1] > g->zh[k]))
                return fail(KL_ERR_INVALID_ARG, "zh must increase strictly");
    if (g->extent <= 0 || g->extent >= (int64_t(1) << 31))
        return fail(KL_ERR_BOUNDS, "extent must be in [1, 2^31)");
    int64_t G = g->g;
    if (g->sj < g->nx + 2 * G) return fail(KL_ERR_BOUNDS, "sj smaller than a padded row");
    if (g->sk < g->sj * (g->ny + 2 * G)) return fail(KL_ERR_BOUNDS, "sk smaller than a padded plane");
    if (g->origin < 0) return fail(KL_ERR_BOUNDS, "origin < 0");
    int64_t z0 = g->origin / g->sk, r = g->origin % g->sk;
    int64_t y0 = r / g->sj, x0 = r % g->sj;
    if (x0 < G || x0 + g->nx + G > g->sj) return fail(KL_ERR_BOUNDS, "x ghosts fall outside a row");
    if (y0 < G || (y0 + g->ny + G) * g->sj > g->sk)
        return fail(KL_ERR_BOUNDS, "y ghosts fall outside a plane");
    if (z0 < G || (z0 + g->nz + G) * g->sk > g->extent)
        return fail(KL_ERR_BOUNDS, "z ghosts fall outside the buffer extent");
    if (geo) {
        geo->x0 = x0;
        geo->y0 = y0;
        geo->z0 = z0;
    }
    return KL_OK;
}

// Vertical metric on levels k in [-g, nz+g): dz_k = zh_{k+1} - zh_k,
// z_k = (zh_k + zh_{k+1})/2, dzh_k = z_k - z_{k-1}; ghost faces mirrored about
// the walls (zbc 1) or wrapped by the domain height (zbc 0).
void zprofile_host(int nz, int g, int zbc, const double *zh, double dz_uniform,
                   std::vector<double> *dzi, std::vector<double> *dzhi)
{
    int n = nz + 2 * g;
    dzi->assign(n, 0.0);
    dzhi->assign(n, 0.0);
    if (!zh) {
        for (int q = 0; q < n; ++q) (*dzi)[q] = (*dzhi)[q] = 1.0 / dz_uniform;
        return;
    }
    double L = zh[nz] - zh[0];
    auto face = [&](int k) -> double {
        if (k >= 0 && k <= nz) return zh[k];
        if (zbc == 1) return k < 0 ? 2.0 * zh[0] - zh[-k] : 2.0 * zh[nz] - zh[2 * nz - k];
        return k < 0 ? zh[k + nz] - L : zh[k - nz] + L;
    };
    auto centre = [&](int k) { return 0.5 * (face(k) + face(k + 1)); };
    for (int k = -g; k < nz + g; ++k) {
        (*dzi)[k + g] = 1.0 / (face(k + 1) - face(k));
        (*dzhi)[k + g] = 1.0 / (centre(k) - centre(k - 1));
    }
}

}  // namespace kl
