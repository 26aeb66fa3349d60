// compile.cpp -- float64 host compiler: elementary sequences (§4.1) -> device program.
//
// The paper's master process precomputes every spin-independent term once (§6.3), e.g. the
// trigonometric functions of the RF pulses of Eq. 3.19; this is that step.  All arithmetic
// here is float64; the float32 program receives (hi, lo) float pairs where one float would
// lose phase accuracy (gradient moments, interval lengths).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>
#include <string>
#include <vector>

#include "../../include/mrsim.h"
#include "compiled.h"

namespace mrsim {

namespace {

// One lowered event.  Members that no kind uses together share storage, 56 bytes in all: every
// pass of the compiler streams the item list, and much of the compile time is spent moving it.
// Each member is read only for the kinds that write it.
struct Item {
    double k[3];  // PREC, SAMPLE: gradient moment γ/2π·G·Δt [cycles/m]
    union {
        double dt;     // PREC, SAMPLE: interval [s]
        double alpha;  // RF: flip angle
    };
    union {
        int64_t j;   // SAMPLE: sample index; SNAP: snapshot index
        double phi;  // RF: phase
    };
    union {
        double adc_phase;  // SAMPLE: receiver phase
        double tau;        // RF, END, SNAP: time since the previous RF pulse [s]
    };
    int32_t param;  // RF: learnable-flip index of a parametric pulse, or -1
    enum Kind : int32_t { RF, PREC, SAMPLE, END, SNAP } kind;
};
static_assert(sizeof(Item) == 56, "Item layout");

using Key = std::array<uint64_t, 4>;

Key key_of(const double k[3], double dt) {
    Key key;
    double v[4] = {k[0], k[1], k[2], dt};
    for (int i = 0; i < 4; ++i) {
        double x = v[i] == 0.0 ? 0.0 : v[i];  // fold -0 into +0
        std::memcpy(&key[i], &x, 8);
    }
    return key;
}

struct KeyHash {
    size_t operator()(const Key &k) const {
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (uint64_t v : k) h = (h ^ v) * 0xBF58476D1CE4E5B9ull;
        return (size_t)(h ^ (h >> 31));
    }
};

bool is_zero(const double k[3], double dt) { return k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0 && dt == 0.0; }

uint64_t bits(double x) {
    uint64_t b;
    x = x == 0.0 ? 0.0 : x;
    std::memcpy(&b, &x, 8);
    return b;
}

// Top-`limit` keys by use count (count >= 2), ties broken by first appearance.
template <class K, class UseMap>
std::map<K, int> pick_classes(const UseMap &uses, int limit) {
    std::vector<std::pair<K, std::pair<int64_t, int64_t>>> v(uses.begin(), uses.end());
    std::sort(v.begin(), v.end(), [](const auto &a, const auto &b) {
        if (a.second.first != b.second.first) return a.second.first > b.second.first;
        return a.second.second < b.second.second;
    });
    std::map<K, int> out;
    for (auto &kv : v) {
        if ((int)out.size() >= limit || kv.second.first < 2) break;
        int id = (int)out.size();
        out[kv.first] = id;
    }
    return out;
}

// cos and sin of x, remembered for repeated arguments: shaped pulses repeat their flip angles
// every TR and the receiver phase is constant along a readout, so most calls are lookups.
class TrigCache {
    struct Entry {
        uint64_t key;
        double c, s;
        bool ok;
    };
    static constexpr size_t N = 4096;
    std::vector<Entry> t_;
    const Entry *last_ = nullptr;

  public:
    TrigCache() : t_(N, Entry{0, 0.0, 0.0, false}) {}
    void get(double x, double &c, double &s) {
        uint64_t b;
        std::memcpy(&b, &x, 8);
        if (last_ && last_->key == b) {  // a readout repeats its receiver phase sample after sample
            c = last_->c;
            s = last_->s;
            return;
        }
        Entry &e = t_[(b ^ (b >> 23) ^ (b >> 41)) & (N - 1)];
        last_ = &e;
        if (!(e.ok && e.key == b)) e = Entry{b, std::cos(x), std::sin(x), true};
        c = e.c;
        s = e.s;
    }
};

struct Group {
    size_t first;
    int64_t n;  // number of items (samples for runs)
};

// Per-thread scratch for the lowered items and their groups: kept between calls, so that
// compiling sequences of similar size touches no fresh pages (above 64 MB it is released).
struct Scratch {
    std::vector<Item> items;
    std::vector<Group> groups;
};
constexpr size_t SCRATCH_KEEP_BYTES = size_t(64) << 20;
struct ScratchLease {
    Scratch &s;
    ScratchLease() : s(get()) {
        s.items.clear();
        s.groups.clear();
    }
    ~ScratchLease() {
        if (s.items.capacity() * sizeof(Item) + s.groups.capacity() * sizeof(Group) > SCRATCH_KEEP_BYTES) {
            std::vector<Item>().swap(s.items);
            std::vector<Group>().swap(s.groups);
        }
    }
    static Scratch &get() {
        static thread_local Scratch t;
        return t;
    }
};

// Use counts of class keys: key -> (count, first position); consecutive uses of one key (the
// sub-pulses of a shaped pulse, the samples of a readout) skip the hash lookup.
template <class K, class H = std::hash<K>>
struct Uses {
    using Map = std::unordered_map<K, std::pair<int64_t, int64_t>, H>;
    Map m;
    typename Map::iterator last = m.end();
    void add(const K &key, int64_t cnt, int64_t pos) {
        if (last != m.end() && last->first == key) {
            last->second.first += cnt;
            return;
        }
        auto r = m.try_emplace(key, cnt, pos);
        if (!r.second) r.first->second.first += cnt;
        last = r.first;
    }
    int64_t count(const K &key) const {
        auto f = m.find(key);
        return f == m.end() ? 0 : f->second.first;
    }
};

// Class index of a key (-1: none), remembering the previous query: consecutive items mostly ask
// for the same key.
template <class K>
struct ClassOf {
    const std::map<K, int> &map;
    K last{};
    int last_id = -1;
    bool valid = false;
    explicit ClassOf(const std::map<K, int> &m) : map(m) {}
    int operator()(const K &key) {
        if (!(valid && key == last)) {
            auto f = map.find(key);
            last = key;
            last_id = f == map.end() ? -1 : f->second;
            valid = true;
        }
        return last_id;
    }
};

// Compensated running sum (Neumaier's variant of Kahan summation): the rounding error of each
// addition is carried in `c`, so an interval made of many short events (a list on a fine time
// raster) sums to its moment within about one rounding instead of one per event.  For one or two
// terms the value equals the plain sum.
struct CSum {
    double s = 0.0, c = 0.0;
    void set(double x) {  // the first term: value() is the same as for add() to an empty sum
        s = x;
        c = 0.0;
    }
    void add(double x) {
        const double t = s + x;
        c += std::fabs(s) >= std::fabs(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

bool same_interval(const Item &a, const Item &b) {  // the key equality of key_of, without the keys
    return a.k[0] == b.k[0] && a.k[1] == b.k[1] && a.k[2] == b.k[2] && a.dt == b.dt;
}

void split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

}  // namespace

int compile_sequence(const mrsim_event *ev, int64_t n, double gamma_hz, Compiled &out, std::string &err,
                     int64_t n_snap, const int64_t *snap_after, const int32_t *rf_param, int32_t n_params) {
    out = Compiled();
    if (rf_param && (n_params < 0 || n_params > TRAIN_TABLE_MAX / 2)) {
        err = "parametric pulses: n_params must be in [0, " + std::to_string(TRAIN_TABLE_MAX / 2) + "]";
        return MRSIM_EINVAL;
    }
    if (n_snap < 0 || (n_snap > 0 && !snap_after)) {
        err = "invalid snapshot list";
        return MRSIM_EINVAL;
    }
    for (int64_t q = 0; q < n_snap; ++q)
        if (snap_after[q] < 0 || snap_after[q] >= n || (q > 0 && snap_after[q] <= snap_after[q - 1])) {
            err = "snapshot " + std::to_string(q) + ": event indices must be strictly increasing and < n_events";
            return MRSIM_EINVAL;
        }
    if (!(gamma_hz > 0.0) || !std::isfinite(gamma_hz)) {
        err = "gamma_hz_per_t must be finite and > 0";
        return MRSIM_EINVAL;
    }
    if (n < 0 || (n > 0 && !ev)) {
        err = "invalid event array";
        return MRSIM_EINVAL;
    }
    // ---- validate and lower to items -------------------------------------------------------
    ScratchLease lease;
    std::vector<Item> &items = lease.s.items;
    items.reserve((size_t)n + 2);
    double tau = 0.0;
    // The pending free interval pk since the last item.  Its trailing events that share one
    // gradient tg are also summed on their own (tk), with hk the pending interval before them: a
    // sample whose event has that gradient absorbs the trailing part (one interval of constant
    // gradient; precession and relaxation compose), so a readout whose dwell is split into several
    // events still compiles to uniform samples.
    // (moments and durations as compensated sums: components 0-2 the moment, 3 the duration;
    // each sum holds a value only while its flag is set)
    bool have = false, hhave = false, thave = false;
    CSum pk[4], hk[4], tk[4];
    double tg[3] = {0, 0, 0};
    int64_t j = 0, snap_next = 0;
    auto push_prec = [&](const CSum *sum) {
        const double k[3] = {sum[0].value(), sum[1].value(), sum[2].value()}, dt = sum[3].value();
        if (is_zero(k, dt)) return;
        Item &it = items.emplace_back();
        it.kind = Item::PREC;
        std::memcpy(it.k, k, sizeof k);
        it.dt = dt;
    };
    auto reset = [&]() { have = hhave = thave = false; };
    auto flush = [&]() {
        if (have) push_prec(pk);
        reset();
    };
    auto same_g = [&](const mrsim_event &e) { return thave && e.gx == tg[0] && e.gy == tg[1] && e.gz == tg[2]; };
    for (int64_t i = 0; i < n; ++i) {
        const mrsim_event &e = ev[i];
        const double f[7] = {e.dt, e.gx, e.gy, e.gz, e.rf_flip, e.rf_phase, e.adc_phase};
        for (double v : f)
            if (!std::isfinite(v)) {
                err = "event " + std::to_string(i) + ": non-finite field";
                return MRSIM_EINVAL;
            }
        if (e.dt < 0.0) {
            err = "event " + std::to_string(i) + ": negative duration";
            return MRSIM_EINVAL;
        }
        if ((e.adc != 0 && e.adc != 1) || e.reserved != 0) {
            err = "event " + std::to_string(i) + ": adc must be 0/1 and reserved 0";
            return MRSIM_EINVAL;
        }
        const int32_t prm = rf_param ? rf_param[i] : -1;
        if (prm < -1 || prm >= (rf_param ? n_params : 0)) {
            err = "event " + std::to_string(i) + ": learnable-flip index out of range";
            return MRSIM_EINVAL;
        }
        if (e.rf_flip != 0.0 || prm >= 0) {
            flush();
            Item &it = items.emplace_back();
            it.kind = Item::RF;
            it.alpha = e.rf_flip;
            it.phi = e.rf_phase;
            it.tau = tau;
            it.param = prm;
            tau = 0.0;
        }
        const double k[3] = {gamma_hz * e.gx * e.dt, gamma_hz * e.gy * e.dt, gamma_hz * e.gz * e.dt};
        if (e.adc) {
            double sk[3], sdt;
            if (same_g(e)) {  // the trailing constant-gradient part joins the sample's interval
                if (hhave) push_prec(hk);
                for (int c = 0; c < 4; ++c) tk[c].add(c < 3 ? k[c] : e.dt);
                for (int c = 0; c < 3; ++c) sk[c] = tk[c].value();
                sdt = tk[3].value();
                reset();
            } else {
                flush();
                std::memcpy(sk, k, sizeof k);
                sdt = e.dt;
            }
            Item &it = items.emplace_back();
            it.kind = Item::SAMPLE;
            std::memcpy(it.k, sk, sizeof sk);
            it.dt = sdt;
            it.j = j++;
            it.adc_phase = e.adc_phase;
        } else {
            const bool fresh = !same_g(e);
            if (fresh) {  // a new trailing run starts here
                if (have)
                    for (int c = 0; c < 4; ++c) hk[c] = pk[c];
                hhave = have;
                tg[0] = e.gx;
                tg[1] = e.gy;
                tg[2] = e.gz;
                thave = true;
            }
            for (int c = 0; c < 4; ++c) {
                const double v = c < 3 ? k[c] : e.dt;
                if (fresh)
                    tk[c].set(v);
                else
                    tk[c].add(v);
                if (have)
                    pk[c].add(v);
                else
                    pk[c].set(v);
            }
            have = true;
        }
        tau += e.dt;
        if (snap_next < n_snap && snap_after[snap_next] == i) {  // state after event i
            flush();
            Item &it = items.emplace_back();
            it.kind = Item::SNAP;
            it.j = snap_next++;
            it.tau = tau;
            tau = 0.0;  // the snapshot applies the T1 recovery so far
        }
    }
    flush();
    {
        Item &it = items.emplace_back();
        it.kind = Item::END;
        it.tau = tau;
    }
    out.n_adc = j;
    out.n_snap = n_snap;

    // ---- group sample runs and count class uses -------------------------------------------------
    std::vector<Group> &groups = lease.s.groups;
    groups.resize(items.size());
    size_t n_groups = 0;
    for (size_t i = 0; i < items.size();) {
        if (items[i].kind == Item::SAMPLE && !is_zero(items[i].k, items[i].dt)) {
            size_t e = i + 1;
            while (e < items.size() && items[e].kind == Item::SAMPLE && (int64_t)(e - i) < RUN_MAX &&
                   same_interval(items[e], items[i]))
                ++e;
            groups[n_groups++] = {i, (int64_t)(e - i)};
            i = e;
        } else {
            groups[n_groups++] = {i, 1};
            ++i;
        }
    }
    groups.resize(n_groups);
    Uses<Key, KeyHash> puses;
    Uses<uint64_t> e1uses, e2uses;
    auto anchor_key = [&](const Item &it, int64_t cnt) {
        double k[3] = {it.k[0] * (double)cnt, it.k[1] * (double)cnt, it.k[2] * (double)cnt};
        return key_of(k, it.dt * (double)cnt);
    };
    auto is_run = [&](size_t g) {
        const Item &it = items[groups[g].first];
        return it.kind == Item::SAMPLE && !is_zero(it.k, it.dt) && groups[g].n >= 4;
    };
    for (size_t g = 0; g < groups.size(); ++g) {
        const Item &it = items[groups[g].first];
        const int64_t pos = (int64_t)groups[g].first;
        if (it.kind == Item::PREC || (it.kind == Item::SAMPLE && !is_zero(it.k, it.dt)))
            puses.add(key_of(it.k, it.dt), groups[g].n, pos);
        if ((it.kind == Item::RF || it.kind == Item::END || it.kind == Item::SNAP) && it.tau > 0.0)
            e1uses.add(bits(it.tau), 1, pos);
    }
    // Rewound readouts: a one-off precession A (phase encoding), a sample run R and a one-off
    // precession B whose moments add up to one that recurs (B undoes A's encoding, as in every
    // Cartesian gradient echo).  Precessions about z commute, so the state after B is the state
    // before A times the phasor of the whole interval A+R+B (Eqs. 3.5, 3.14): the run starts with
    // A inline, its anchor restores from the state before A with that class, and B disappears.
    // Moment components that cancel to rounding level are snapped to zero so that the sum is
    // the same in every repetition.
    auto single = [&](size_t g) {
        const Item &it = items[groups[g].first];
        if (it.kind != Item::PREC) return false;
        return puses.count(key_of(it.k, it.dt)) < 2;  // stays inline
    };
    std::unordered_map<size_t, Key> fkey;  // candidate run group -> key of A+R+B
    std::vector<char> claimed(groups.size(), 0);
    Uses<Key, KeyHash> fuses;
    for (size_t g = 1; g + 1 < groups.size(); ++g) {
        if (claimed[g - 1] || !is_run(g) || !single(g - 1) || !single(g + 1)) continue;
        const Item &A = items[groups[g - 1].first], &R = items[groups[g].first], &B = items[groups[g + 1].first];
        const double n = (double)groups[g].n;
        double k[3];
        for (int c = 0; c < 3; ++c) {
            const double s = A.k[c] + R.k[c] * n + B.k[c];
            const double mag = std::fabs(A.k[c]) + std::fabs(R.k[c] * n) + std::fabs(B.k[c]);
            k[c] = std::fabs(s) <= mag * 0x1p-46 ? 0.0 : s;
        }
        fkey[g] = key_of(k, A.dt + R.dt * n + B.dt);
        claimed[g - 1] = claimed[g + 1] = 1;
        fuses.add(fkey[g], 1, (int64_t)groups[g].first);
    }
    auto recurring = [&](size_t g) {
        auto f = fkey.find(g);
        return f != fkey.end() && fuses.count(f->second) >= 2;
    };
    for (size_t g = 0; g < groups.size(); ++g) {
        if (!is_run(g)) continue;
        if (recurring(g))
            puses.add(fkey[g], 1, (int64_t)groups[g].first);
        else
            puses.add(anchor_key(items[groups[g].first], groups[g].n), 1, (int64_t)groups[g].first);
    }
    auto pmap = pick_classes<Key>(puses.m, MAX_PCLS);
    auto e1map = pick_classes<uint64_t>(e1uses.m, MAX_E1CLS);
    // fused triples: A goes into the run op (role 1), B is dropped (role 2)
    std::vector<char> fused(groups.size(), 0), role(groups.size(), 0);
    for (auto &fk : fkey) {
        const size_t g = fk.first;
        const Item &R = items[groups[g].first];
        if (recurring(g) && pmap.count(fk.second) && pmap.count(key_of(R.k, R.dt))) {
            fused[g] = 1;
            role[g - 1] = 1;
            role[g + 1] = 2;
        }
    }
    // E2 classes: intervals of the precessions that stay inline
    ClassOf<Key> pclass(pmap);
    for (size_t g = 0; g < groups.size(); ++g) {
        const Item &it = items[groups[g].first];
        if ((it.kind == Item::PREC || it.kind == Item::SAMPLE) && !is_zero(it.k, it.dt) && it.dt > 0.0 &&
            pclass(key_of(it.k, it.dt)) < 0 && role[g] != 2)
            e2uses.add(bits(it.dt), groups[g].n, (int64_t)groups[g].first);
    }
    auto e2map = pick_classes<uint64_t>(e2uses.m, MAX_E2CLS);

    out.n_pcls = (int)pmap.size();
    out.n_e1 = (int)e1map.size();
    out.n_e2 = (int)e2map.size();
    out.pcls.assign(4 * (size_t)out.n_pcls, 0.0);
    for (auto &kv : pmap)
        for (int c = 0; c < 4; ++c) std::memcpy(&out.pcls[4 * (size_t)kv.second + c], &kv.first[c], 8);
    out.e1.assign((size_t)out.n_e1, 0.0);
    for (auto &kv : e1map) std::memcpy(&out.e1[(size_t)kv.second], &kv.first, 8);
    out.e2.assign((size_t)out.n_e2, 0.0);
    for (auto &kv : e2map) std::memcpy(&out.e2[(size_t)kv.second], &kv.first, 8);

    // ---- emit ------------------------------------------------------------------------------------
    // Mirrors of the kernel's state: the frame angle ψ (phase of the latest pulse) and the
    // register caches of the phasor class and the T1 class.
    double psi = 0.0;
    int pcache = -1, e1cache = -1;
    out.demod.assign(2 * (size_t)out.n_adc, 0.0);
    auto new32 = [](uint8_t kind) {
        OpF32 o;
        std::memset(&o, 0, sizeof o);
        o.kind = kind;
        o.pcls = o.ecls = o.acls = -1;
        o.adc0 = -1;
        o.n = 1;
        return o;
    };
    auto new64 = [](uint8_t kind) {
        OpF64 o;
        std::memset(&o, 0, sizeof o);
        o.kind = kind;
        o.pcls = o.ecls = o.acls = -1;
        o.adc0 = -1;
        o.n = 1;
        return o;
    };
    auto both = [](OpF32 &a, OpF64 &b, uint16_t fl) {
        a.flags |= fl;
        b.flags |= fl;
    };
    TrigCache trig;
    auto demod = [&](int64_t jj, double adc_phase) {
        // sample sum in the frame ψ: Σ(u + jv) = e^{-jψ} Σ(Mx + jMy), so the factor is e^{-j(φ_adc - ψ)}
        double c, sn;
        trig.get(adc_phase - psi, c, sn);
        out.demod[2 * (size_t)jj] = c;
        out.demod[2 * (size_t)jj + 1] = -sn;
    };
    ClassOf<uint64_t> e1class(e1map);
    auto set_e1 = [&](OpF32 &a, OpF64 &b, double t) {
        if (t > 0.0) {
            const int c = e1class(bits(t));
            if (c >= 0) {
                both(a, b, F_E1CLS);
                a.ecls = b.ecls = (int16_t)c;
                if (e1cache != c) {
                    both(a, b, F_E1LOAD);
                    e1cache = c;
                }
            } else {
                both(a, b, F_E1INL);
            }
        }
        a.f[10] = (float)t;
        b.f[10] = t;
    };
    auto use_pcls = [&](OpF32 &a, OpF64 &b, int c) {
        both(a, b, F_PCLS);
        a.pcls = b.pcls = (int16_t)c;
        if (pcache != c) {
            both(a, b, F_PLOAD);
            pcache = c;
        }
    };
    auto set_inline_prec = [&](OpF32 &a, OpF64 &b, const Item &it) {
        both(a, b, F_INLINE);
        uint16_t terms = (it.k[0] != 0.0 ? F_KX : 0) | (it.k[1] != 0.0 ? F_KY : 0) |
                         (it.k[2] != 0.0 ? F_KZ : 0) | (it.dt != 0.0 ? F_DT : 0);
        both(a, b, terms);
        for (int c = 0; c < 3; ++c) {
            split(it.k[c], a.f[2 * c], a.f[2 * c + 1]);
            b.f[c] = it.k[c];
        }
        split(it.dt, a.f[6], a.f[7]);
        a.f[8] = (float)it.dt;
        b.f[3] = it.dt;
        auto e2 = e2map.find(bits(it.dt));
        if (it.dt > 0.0 && e2 != e2map.end()) {
            both(a, b, F_E2CLS);
            a.ecls = b.ecls = (int16_t)e2->second;
        }
    };
    // Sub-pulse trains (Eq. 3.23): a run of 2..RUN_MAX consecutive fast sub-pulses becomes one
    // OP_RF_TRAIN over a table of (cos α, sin α) pairs; identical runs (the same shaped pulse
    // every TR) share table entries.  Fast sub-pulses wait in `pend` until their run ends.
    std::vector<OpF32> pend32;
    std::vector<OpF64> pend64;
    std::map<std::vector<uint64_t>, int> seen;
    std::vector<uint64_t> tkey;
    if (rf_param) {  // entries 0 .. n_params-1: the learnable flips, written before each launch
        out.train.reserve(2 * (size_t)n_params);
        for (int32_t q = 0; q < n_params; ++q) {
            out.train.push_back(1.0);
            out.train.push_back(0.0);
        }
    }
    // a run of parametric sub-pulses with consecutive indices reads its table entries in place
    auto param_run = [&]() {
        if (!(pend32[0].flags & F_RFTAB)) return -1;
        for (size_t q = 0; q < pend32.size(); ++q)
            if (!(pend32[q].flags & F_RFTAB) || pend32[q].tab != pend32[0].tab + (int)q) return -1;
        return (int)pend32[0].tab;
    };
    auto flush_train = [&]() {
        const size_t n = pend32.size();
        bool mixed = false;
        for (size_t q = 1; q < n; ++q) mixed |= ((pend32[q].flags ^ pend32[0].flags) & F_RFTAB) != 0;
        if (n >= 2 && (pend32[0].flags & F_RFTAB) && !mixed) {
            const int off = param_run();
            if (off >= 0) {
                OpF32 a = pend32[0];
                OpF64 b = pend64[0];
                a.kind = b.kind = OP_RF_TRAIN;
                a.flags = b.flags = (uint16_t)(a.flags & ~F_RFTAB);
                a.n = b.n = (int32_t)n;
                a.adc0 = b.adc0 = off;
                out.ops32.push_back(a);
                out.ops64.push_back(b);
                pend32.clear();
                pend64.clear();
                return;
            }
        } else if (n >= 2 && !mixed) {
            tkey.clear();
            for (size_t q = 0; q < n; ++q) {
                tkey.push_back(bits(pend64[q].f[0]));
                tkey.push_back(bits(pend64[q].f[1]));
            }
            auto it = seen.find(tkey);
            int off = -1;
            if (it != seen.end()) {
                off = it->second;
            } else if ((int64_t)(out.train.size() / 2 + n) <= TRAIN_TABLE_MAX) {
                off = (int)(out.train.size() / 2);
                for (size_t q = 0; q < n; ++q) {
                    out.train.push_back(pend64[q].f[0]);
                    out.train.push_back(pend64[q].f[1]);
                }
                seen.emplace(tkey, off);
            }
            if (off >= 0) {
                OpF32 a = pend32[0];
                OpF64 b = pend64[0];
                a.kind = b.kind = OP_RF_TRAIN;
                a.n = b.n = (int32_t)n;
                a.adc0 = b.adc0 = off;
                out.ops32.push_back(a);
                out.ops64.push_back(b);
                pend32.clear();
                pend64.clear();
                return;
            }
        }
        out.ops32.insert(out.ops32.end(), pend32.begin(), pend32.end());
        out.ops64.insert(out.ops64.end(), pend64.begin(), pend64.end());
        pend32.clear();
        pend64.clear();
    };
    auto push = [&](const OpF32 &a, const OpF64 &b) {
        if (a.kind == OP_RF_FAST) {
            pend32.push_back(a);
            pend64.push_back(b);
            if ((int64_t)pend32.size() == RUN_MAX) flush_train();
            return;
        }
        flush_train();
        out.ops32.push_back(a);
        out.ops64.push_back(b);
    };

    for (size_t g = 0; g < groups.size(); ++g) {
        const Item &it = items[groups[g].first];
        switch (it.kind) {
        case Item::RF: {
            OpF32 a = new32(OP_RF);
            OpF64 b = new64(OP_RF);
            if (it.phi != psi) {
                // turn the frame from ψ to φ: (u + jv) <- (u + jv)·exp(-jδ), δ = φ - ψ; the float32
                // program gets (hi, lo) pairs so that the frame never drifts (it is uniform over spins)
                double cd, sd;
                trig.get(it.phi - psi, cd, sd);
                both(a, b, F_FRAME);
                split(cd, a.f[2], a.f[3]);
                split(sd, a.f[4], a.f[5]);
                b.f[2] = cd;
                b.f[3] = sd;
                psi = it.phi;
            }
            set_e1(a, b, it.tau);
            double ca, sa;
            trig.get(it.alpha, ca, sa);
            a.f[0] = (float)ca;
            a.f[1] = (float)sa;
            b.f[0] = ca;
            b.f[1] = sa;
            if (it.param >= 0) {  // the rotation comes from table entry `param` at run time
                both(a, b, F_RFTAB);
                a.tab = b.tab = (int16_t)it.param;
            }
            // fuse a following class precession (the sub-pulse trains of shaped pulses, Eq. 3.23)
            if (g + 1 < groups.size()) {
                const Item &nx = items[groups[g + 1].first];
                if (nx.kind == Item::PREC) {
                    const int pc = pclass(key_of(nx.k, nx.dt));
                    if (pc >= 0) {
                        use_pcls(a, b, pc);
                        ++g;
                    }
                }
            }
            const uint16_t fast_mask = F_FRAME | F_E1LOAD | F_E1INL | F_PLOAD | F_ADC;
            if ((a.flags & F_E1CLS) && (a.flags & F_PCLS) && !(a.flags & fast_mask)) a.kind = b.kind = OP_RF_FAST;
            push(a, b);
            break;
        }
        case Item::PREC: {
            if (role[g]) break;  // inside a rewound readout: emitted with (A) or absorbed by (B) the run
            OpF32 a = new32(OP_PREC);
            OpF64 b = new64(OP_PREC);
            const int pc = pclass(key_of(it.k, it.dt));
            if (pc >= 0)
                use_pcls(a, b, pc);
            else
                set_inline_prec(a, b, it);
            push(a, b);
            break;
        }
        case Item::SAMPLE: {
            const int64_t cnt = groups[g].n;
            for (int64_t q = 0; q < cnt; ++q) {
                const Item &s = items[groups[g].first + (size_t)q];
                demod(s.j, s.adc_phase);
            }
            if (is_zero(it.k, it.dt)) {
                OpF32 a = new32(OP_PREC);
                OpF64 b = new64(OP_PREC);
                both(a, b, F_ADC);
                a.adc0 = b.adc0 = (int32_t)it.j;
                push(a, b);
                break;
            }
            const int pc = pclass(key_of(it.k, it.dt));
            if (pc >= 0 && cnt > 1) {
                OpF32 a = new32(OP_RUN);
                OpF64 b = new64(OP_RUN);
                use_pcls(a, b, pc);
                a.n = b.n = (int32_t)cnt;
                a.adc0 = b.adc0 = (int32_t)it.j;
                if (fused[g]) {  // A first, then the samples; the anchor covers A, the run and B
                    set_inline_prec(a, b, items[groups[g - 1].first]);
                    both(a, b, F_ANCHOR);
                    a.acls = b.acls = (int16_t)pmap.at(fkey.at(g));
                } else if (cnt >= 4) {
                    auto an = pmap.find(anchor_key(it, cnt));
                    if (an != pmap.end()) {
                        both(a, b, F_ANCHOR);
                        a.acls = b.acls = (int16_t)an->second;
                    }
                }
                push(a, b);
            } else {
                for (int64_t q = 0; q < cnt; ++q) {
                    const Item &s = items[groups[g].first + (size_t)q];
                    OpF32 a = new32(OP_PREC);
                    OpF64 b = new64(OP_PREC);
                    if (pc >= 0)
                        use_pcls(a, b, pc);
                    else
                        set_inline_prec(a, b, s);
                    both(a, b, F_ADC);
                    a.adc0 = b.adc0 = (int32_t)s.j;
                    push(a, b);
                }
            }
            break;
        }
        case Item::SNAP: {
            OpF32 a = new32(OP_SNAP);
            OpF64 b = new64(OP_SNAP);
            set_e1(a, b, it.tau);
            double cp, sp;
            trig.get(psi, cp, sp);
            a.f[0] = (float)cp;
            a.f[1] = (float)sp;
            b.f[0] = cp;
            b.f[1] = sp;
            a.adc0 = b.adc0 = (int32_t)it.j;
            push(a, b);
            break;
        }
        case Item::END: {
            OpF32 a = new32(OP_END);
            OpF64 b = new64(OP_END);
            set_e1(a, b, it.tau);
            // back to the laboratory frame for the final state: (Mx + jMy) = (u + jv)·exp(+jψ)
            double cp, sp;
            trig.get(psi, cp, sp);
            a.f[0] = (float)cp;
            a.f[1] = (float)sp;
            b.f[0] = cp;
            b.f[1] = sp;
            push(a, b);
            break;
        }
        }
    }
    flush_train();
    if (out.n_adc > (int64_t)INT32_MAX) {
        err = "too many ADC samples";
        return MRSIM_EINVAL;
    }
    // Train maps: trains that recur TRAIN_MAP_MIN times or more with the same classes and table
    // entries (the same shaped pulse in every TR) get a map kind, in order of first appearance.
    // A train's effect depends only on these and on the spin, so one map per spin and kind stands
    // for every occurrence.  Programs with learnable flips rewrite their table between launches:
    // no maps there.
    if (!rf_param) {
        std::map<std::array<int32_t, 4>, int> count;
        std::vector<std::array<int32_t, 4>> order;
        for (const OpF32 &o : out.ops32) {
            if (o.kind != OP_RF_TRAIN || !(o.flags & F_E1CLS) || !(o.flags & F_PCLS)) continue;
            const std::array<int32_t, 4> key = {o.pcls, o.ecls, o.adc0, o.n};
            if (count[key]++ == 0) order.push_back(key);
        }
        std::map<std::array<int32_t, 4>, int> kind;
        for (const auto &key : order) {
            if ((int)kind.size() == TRAIN_MAP_MAX) break;
            if (count[key] < TRAIN_MAP_MIN) continue;
            const int t = (int)kind.size();
            kind.emplace(key, t);
            out.tmap.insert(out.tmap.end(), key.begin(), key.end());
        }
        for (size_t i = 0; i < out.ops32.size() && !kind.empty(); ++i) {
            OpF32 &a = out.ops32[i];
            if (a.kind != OP_RF_TRAIN || !(a.flags & F_E1CLS) || !(a.flags & F_PCLS)) continue;
            auto it = kind.find({a.pcls, a.ecls, a.adc0, a.n});
            if (it == kind.end()) continue;
            OpF64 &b = out.ops64[i];
            a.flags = b.flags = (uint16_t)(a.flags | F_TMAP);
            a.tab = b.tab = (int16_t)it->second;
        }
    }
    return MRSIM_OK;
}

}  // namespace mrsim
