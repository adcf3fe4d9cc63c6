// api.cu -- host side of the C ABI declared in include/fwi.h: argument
// validation, plans (host memory only), buffer sizing and the entry points.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "fwi_internal.cuh"

namespace fwi {
size_t w2_trace_smem(int nt, int nxi);
}

using fwi::Plan;

namespace {

thread_local char g_err[512] = "";

fwi_status fail(fwi_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

fwi_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(FWI_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

const Plan *as_plan(const fwi_plan *p) { return reinterpret_cast<const Plan *>(p); }

// the record planes and checkpoint slots are moved in 16-byte units (vector
// stores and loads, bulk L2 prefetches), the workspace holds them too
bool misaligned16(const void *p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }


}  // namespace

fwi_status fwi::record_error(fwi_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

extern "C" {

const char *fwi_last_error(void) { return g_err; }

int fwi_version(void) { return FWI_VERSION; }

fwi_status fwi_plan_create(const fwi_problem *prob, const fwi_w2_params *w2, fwi_plan **out)
{
    g_err[0] = 0;
    if (!out) return fail(FWI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!prob || !w2) return fail(FWI_ERR_INVALID_ARG, "problem or w2 params is NULL");
    const fwi_problem &p = *prob;
    if (p.nz < 1 || p.nx < 1) return fail(FWI_ERR_INVALID_ARG, "nz, nx must be >= 1");
    if (p.nb < 0) return fail(FWI_ERR_INVALID_ARG, "nb must be >= 0");
    if (p.top_bc != 0 && p.top_bc != 1) return fail(FWI_ERR_INVALID_ARG, "top_bc must be 0 or 1");
    if (p.nt < 2) return fail(FWI_ERR_INVALID_ARG, "nt must be >= 2");
    if (!finite_pos(p.dt) || !finite_pos(p.dx) || !finite_pos(p.dz))
        return fail(FWI_ERR_INVALID_ARG, "dt, dx, dz must be finite and > 0");
    if (p.ns < 1 || p.ns > FWI_MAX_SHOTS)
        return fail(FWI_ERR_INVALID_ARG, "ns must be in [1, %d]", FWI_MAX_SHOTS);
    if (p.nr < 1 || p.nr > FWI_MAX_RECEIVERS)
        return fail(FWI_ERR_INVALID_ARG, "nr must be in [1, %d]", FWI_MAX_RECEIVERS);
    if (!p.src_iz || !p.src_ix || !p.rec_iz || !p.rec_ix)
        return fail(FWI_ERR_INVALID_ARG, "source/receiver index arrays must not be NULL");
    if (p.batch < 1) return fail(FWI_ERR_INVALID_ARG, "batch must be >= 1");
    if (!finite_pos(p.f_peak)) return fail(FWI_ERR_INVALID_ARG, "f_peak must be > 0");
    if (!std::isfinite(p.t0)) return fail(FWI_ERR_INVALID_ARG, "t0 must be finite");
    if (!finite_pos(p.v_ref)) return fail(FWI_ERR_INVALID_ARG, "v_ref must be > 0");
    if (!(p.refl_R > 0.0 && p.refl_R <= 1.0))
        return fail(FWI_ERR_INVALID_ARG, "refl_R must be in (0, 1]");
    if (!finite_pos(p.v_max)) return fail(FWI_ERR_INVALID_ARG, "v_max must be > 0");
    if (p.checkpoint_every < 0) return fail(FWI_ERR_INVALID_ARG, "checkpoint_every must be >= 0");
    if (w2->n_xi < 2) return fail(FWI_ERR_INVALID_ARG, "n_xi must be >= 2");
    if (!(w2->k >= 0.0) || !std::isfinite(w2->k)) return fail(FWI_ERR_INVALID_ARG, "k must be >= 0");
    if (!(w2->cshift_factor >= 0.0) || !std::isfinite(w2->cshift_factor))
        return fail(FWI_ERR_INVALID_ARG, "cshift_factor must be >= 0");
    if (!(w2->eps_density >= 0.0) || !std::isfinite(w2->eps_density))
        return fail(FWI_ERR_INVALID_ARG, "eps_density must be >= 0");
    if (w2->squared != 0 && w2->squared != 1) return fail(FWI_ERR_INVALID_ARG, "squared must be 0 or 1");
    if (p.shape < FWI_SHAPE_DEFAULT || p.shape > FWI_SHAPE_TILED_QUADS)
        return fail(FWI_ERR_INVALID_ARG, "shape %d is not an FWI_SHAPE_* value", p.shape);
    if (p.kernels < FWI_KERNELS_AUTO || p.kernels > FWI_KERNELS_CPML)
        return fail(FWI_ERR_INVALID_ARG, "kernels must be 0 (auto), 1, 2, 3 or 4");
    if (p.absorber != FWI_ABSORBER_SPONGE && p.absorber != FWI_ABSORBER_CPML)
        return fail(FWI_ERR_INVALID_ARG, "absorber must be 0 (sponge) or 1 (CPML)");
    if (p.space_order != 0 && p.space_order != 4 && p.space_order != 8)
        return fail(FWI_ERR_INVALID_ARG, "space_order must be 0, 4 or 8");
    const int order = p.space_order == 8 ? 8 : 4;
    // leapfrog: stable while v dt sqrt(1/dx^2 + 1/dz^2) <= 2 / sqrt(lambda), lambda
    // the largest |symbol| of the 1D second difference at theta = pi:
    // 16/3 at 4th order, 205/72 + 2 (8/5 + 1/5 + 8/315 + 1/560) at 8th order
    const double lambda = order == 8 ? 205.0 / 72 + 2 * (8.0 / 5 + 1.0 / 5 + 8.0 / 315 + 1.0 / 560)
                                     : 16.0 / 3.0;
    const double cfl_max = 2.0 / std::sqrt(lambda);
    const double cfl = (double)p.v_max * p.dt *
                       std::sqrt(1.0 / ((double)p.dx * p.dx) + 1.0 / ((double)p.dz * p.dz));
    if (cfl > cfl_max)
        return fail(FWI_ERR_UNSTABLE_CFL,
                    "v_max dt sqrt(1/dx^2 + 1/dz^2) = %.4f exceeds %.4f (order %d leapfrog)", cfl,
                    cfl_max, order);

    Plan *pl = new (std::nothrow) Plan();
    if (!pl) return fail(FWI_ERR_INVALID_ARG, "out of host memory");
    pl->fwd_pair = false;
    pl->adj_pair = false;
    pl->tiled = false;
    pl->tile_rows = p.shape == FWI_SHAPE_TILED_ROWS4 ? 4 : 8;
    // tiled: float4 column quads unless a scalar row shape is asked for
    pl->tile_quads = p.shape != FWI_SHAPE_TILED_ROWS8 && p.shape != FWI_SHAPE_TILED_ROWS4;
    pl->p = p;
    pl->p.space_order = order;
    pl->w2 = *w2;
    pl->NZ = p.nz + p.nb;
    pl->NX = p.nx + 2 * p.nb;
    pl->t0 = p.t0 > 0.0 ? p.t0 : 1.1 / p.f_peak;
    for (int i = 0; i < p.ns; ++i) {
        if (p.src_iz[i] < 0 || p.src_iz[i] >= p.nz || p.src_ix[i] < 0 || p.src_ix[i] >= p.nx) {
            delete pl;
            return fail(FWI_ERR_INVALID_ARG, "source %d at (%d, %d) is outside the %dx%d grid", i,
                        p.src_iz[i], p.src_ix[i], p.nz, p.nx);
        }
        pl->src_pz[i] = p.src_iz[i];
        pl->src_px[i] = p.src_ix[i] + p.nb;
    }
    for (int i = 0; i < p.nr; ++i) {
        if (p.rec_iz[i] < 0 || p.rec_iz[i] >= p.nz || p.rec_ix[i] < 0 || p.rec_ix[i] >= p.nx) {
            delete pl;
            return fail(FWI_ERR_INVALID_ARG, "receiver %d at (%d, %d) is outside the %dx%d grid", i,
                        p.rec_iz[i], p.rec_ix[i], p.nz, p.nx);
        }
        pl->rec_pz[i] = p.rec_iz[i];
        pl->rec_px[i] = p.rec_ix[i] + p.nb;
    }
    pl->p.src_iz = pl->p.src_ix = pl->p.rec_iz = pl->p.rec_ix = nullptr;
    if (pl->NZ > 32767 || pl->NX > 32767) {
        delete pl;
        return fail(FWI_ERR_UNSUPPORTED, "padded grid %dx%d too large", pl->NZ, pl->NX);
    }
    const int fam = p.kernels;
    // the CPML absorber runs on its own kernels
    pl->cpml = p.absorber == FWI_ABSORBER_CPML;
    pl->ws_c = 0;
    if (pl->cpml || fam == FWI_KERNELS_CPML) {
        const char *need = nullptr;
        if (!pl->cpml) need = "absorber = FWI_ABSORBER_CPML";
        else if (order != 4) need = "space_order 4";
        else if (p.top_bc != 0) need = "top_bc = 0";
        else if (p.checkpoint_every != 0) need = "checkpoint_every = 0";
        else if (fam != FWI_KERNELS_AUTO && fam != FWI_KERNELS_CPML)
            need = "kernels = FWI_KERNELS_AUTO or FWI_KERNELS_CPML";
        else if ((long long)p.batch * p.ns > 65535) need = "batch x ns <= 65535";
        for (int i = 0; !need && i < p.nr; ++i)
            for (int k = 0; k < i; ++k)
                if (pl->rec_px[i] == pl->rec_px[k] && pl->rec_pz[i] == pl->rec_pz[k]) {
                    need = "distinct receiver cells";
                    break;
                }
        if (need) {
            delete pl;
            return fail(FWI_ERR_UNSUPPORTED, "CPML plans (FWI_KERNELS_CPML) need %s", need);
        }
    }
    // the resident kernels implement the 4th-order stencil only
    pl->fast = !pl->cpml && (fam == FWI_KERNELS_AUTO || fam == FWI_KERNELS_RESIDENT) && order == 4 &&
               fwi::fast_bucket(pl->NZ, pl->NX, &pl->fast_P, &pl->fast_PR, &pl->fast_NZM);
    if (pl->fast) {
        const int nstrip = (pl->NZ + fwi::kFastRows - 1) / fwi::kFastRows;
        for (int adj = 0; adj < 2; ++adj) {
            fwi::ResidentShape &sh = adj ? pl->shape_adj : pl->shape;
            sh.rows = fwi::kFastRows;
            sh.maxrows = fwi::kFastRows;
            sh.nstrip = nstrip;
            sh.threads = ((pl->NX * nstrip + 31) / 32) * 32;
            const int chunk = fwi::fast_chunk(pl->fast_P, pl->fast_NZM, adj != 0, p.nr);
            sh.chunk = chunk;
            sh.smem = fwi::fast_smem(pl->fast_P, pl->fast_NZM, adj != 0, chunk, p.nr);
            if (chunk < 1) pl->fast = false;
        }
        pl->nzs = nstrip * fwi::kFastRows;
        pl->fwd_pair = pl->fast && p.shape != FWI_SHAPE_RESIDENT_COLUMNS &&
                       fwi::fwd_pair_ok(pl->NX, pl->NZ, pl->fast_NZM);
        if (pl->fwd_pair) {
            fwi::ResidentShape &sh = pl->shape;
            const int nstrip2 = (pl->NZ + fwi::kFastRows / 2 - 1) / (fwi::kFastRows / 2);
            sh.rows = fwi::kFastRows / 2;
            sh.maxrows = sh.rows;
            sh.nstrip = nstrip2;
            sh.threads = (((pl->NX / 2) * nstrip2 + 31) / 32) * 32;
            const int chunk = fwi::fast_chunk(fwi::kPairPitch, pl->fast_NZM, false, p.nr);
            sh.chunk = chunk;
            sh.smem = fwi::fast_smem(fwi::kPairPitch, pl->fast_NZM, false, chunk, p.nr);
            if (chunk < 1) pl->fwd_pair = false;
            if (nstrip2 * sh.rows > pl->nzs) pl->nzs = nstrip2 * sh.rows;
        }
        if (pl->fwd_pair) {   // the adjoint on the same column pairs
            fwi::ResidentShape sh = pl->shape;
            const int chunk = fwi::fast_chunk(fwi::kPairPitch, pl->fast_NZM, true, p.nr);
            sh.chunk = chunk;
            sh.smem = fwi::fast_smem(fwi::kPairPitch, pl->fast_NZM, true, chunk, p.nr);
            if (chunk >= 1) {
                pl->shape_adj = sh;
                pl->adj_pair = true;
            }
        }
        if (!pl->fwd_pair && pl->fast) {   // restore the single-column forward shape
            fwi::ResidentShape &sh = pl->shape;
            sh.rows = fwi::kFastRows;
            sh.maxrows = fwi::kFastRows;
            sh.nstrip = nstrip;
            sh.threads = ((pl->NX * nstrip + 31) / 32) * 32;
            const int chunk = fwi::fast_chunk(pl->fast_P, pl->fast_NZM, false, p.nr);
            sh.chunk = chunk;
            sh.smem = fwi::fast_smem(pl->fast_P, pl->fast_NZM, false, chunk, p.nr);
        }
    }
    if (pl->cpml) pl->nzs = pl->NZ;
    if (!pl->fast && !pl->cpml) {
        pl->nzs = pl->NZ;
        if (fam == FWI_KERNELS_TILED || fam == FWI_KERNELS_CLUSTER || order == 8 ||
            !fwi::choose_resident_shape(pl->NZ, pl->NX, p.nr, false, &pl->shape) ||
            !fwi::choose_resident_shape(pl->NZ, pl->NX, p.nr, true, &pl->shape_adj)) {
            if (fam == FWI_KERNELS_RESIDENT) {
                delete pl;
                return fail(FWI_ERR_UNSUPPORTED,
                            "the resident kernels hold 4th-order %dx%d padded grids only up to "
                            "one CTA's shared memory",
                            pl->NZ, pl->NX);
            }
            // beyond one CTA's shared memory: global-memory tiled kernels
            // (one launch per step; grid z = models x shots)
            if ((long long)p.batch * p.ns > 65535) {
                delete pl;
                return fail(FWI_ERR_UNSUPPORTED,
                            "batch x ns = %lld exceeds 65535 for the tiled propagator",
                            (long long)p.batch * p.ns);
            }
            pl->tiled = true;
        }
    }
    pl->NXp = (pl->NX + 3) / 4 * 4;
    pl->rec_pitch = pl->fast ? pl->fast_PR : (pl->tiled ? pl->NXp : pl->NX);
    // store-all 4th-order plans of the tiled family run on the cluster kernels
    // when a grid's rows fit a cluster's shared memory
    pl->cluster = false;
    if (pl->tiled && (fam == FWI_KERNELS_AUTO || fam == FWI_KERNELS_CLUSTER) && order == 4 &&
        p.checkpoint_every == 0 && pl->NX + 4 <= fwi::kCluPitch) {
        // rows per thread strip RS (a compile-time bucket), strips per column,
        // rows per CTA RC = nstrip RS and CTAs per cluster C = ceil(NZ / RC).
        // Column pairs (even padded width) first, then single columns of 13 or
        // 19 rows, as far as the requested shape allows.
        const int rc0 = (pl->NZ + fwi::kClusterCTAs - 1) / fwi::kClusterCTAs;
        // static shared memory of the kernels: four mbarriers, a flag, one sum, a TMEM slot
        const size_t limit = 227 * 1024 - 64;
        struct Try { bool pair; int rs; };
        const Try tries[] = {{true, fwi::kCluPairRows}, {false, 13}, {false, 19}};
        for (const Try &t : tries) {
            if (pl->cluster) break;
            if ((p.shape == FWI_SHAPE_CLUSTER_PAIRS && !t.pair) ||
                (p.shape == FWI_SHAPE_CLUSTER_RS13 && (t.pair || t.rs != 13)) ||
                (p.shape == FWI_SHAPE_CLUSTER_RS19 && (t.pair || t.rs != 19)))
                continue;
            if (t.pair && (pl->NX % 2 != 0 || pl->NX + 4 > fwi::kCluPairPitch)) continue;
            const int P = t.pair ? fwi::kCluPairPitch : fwi::kCluPitch;
            const int RS = t.rs;
            const int nstrip = (rc0 + RS - 1) / RS;
            const int threads = ((t.pair ? pl->NX / 2 : pl->NX) * nstrip + 31) / 32 * 32;
            if (threads > (t.pair ? fwi::kCluPairThreads : fwi::clu_max_threads(RS))) continue;
            const int RC = nstrip * RS;
            const int C = (pl->NZ + RC - 1) / RC;
            int chunk[2] = {0, 0};
            if (C >= 2) {
                for (int adj = 0; adj < 2; ++adj) {
                    const size_t fixed = fwi::cluster_smem(RC, P, adj != 0, 0, p.nr, t.pair);
                    const size_t per = ((size_t)p.nr + 1) * 4;
                    size_t c = fixed + per > limit ? 0 : (limit - fixed) / per;
                    chunk[adj] = c > 32 ? 32 : (int)c;
                }
            }
            bool ok = C >= 2 && C <= fwi::kClusterCTAs && chunk[0] >= 1 && chunk[1] >= 1;
            // the adjoint injects each receiver from the thread owning its cell:
            // at most one receiver per column of a strip
            for (int i = 0; ok && i < p.nr; ++i)
                for (int k = 0; k < i; ++k)
                    if (pl->rec_px[i] == pl->rec_px[k] &&
                        pl->rec_pz[i] / RS == pl->rec_pz[k] / RS) {
                        ok = false;
                        break;
                    }
            if (ok) {
                pl->cluster = true;
                pl->clu = fwi::ClusterArgs{P, C, RC, RS, nstrip, pl->NXp, 0, nullptr, nullptr,
                                           0, 0ull, t.pair ? 1 : 0};
                pl->clu_threads = threads;
                pl->clu_chunk_fwd = chunk[0];
                pl->clu_chunk_adj = chunk[1];
                // record: C RC rows per plane at the pitch kCluPitch - 1
                pl->nzs = C * RC;
                pl->rec_pitch = fwi::kCluPitch - 1;
            }
        }
    }
    // the shape must be one of the family the plan runs on
    {
        const int sh = p.shape;
        bool ok = sh == FWI_SHAPE_DEFAULT;
        const char *family = "CPML";
        if (pl->cpml) {
        } else if (pl->fast) {
            family = "resident";
            ok = ok || sh == FWI_SHAPE_RESIDENT_COLUMNS ||
                 (sh == FWI_SHAPE_RESIDENT_PAIRS && pl->fwd_pair);
        } else if (pl->cluster) {
            family = "cluster";
            ok = ok || sh == FWI_SHAPE_CLUSTER_RS13 || sh == FWI_SHAPE_CLUSTER_RS19 ||
                 sh == FWI_SHAPE_CLUSTER_PAIRS;
        } else if (pl->tiled) {
            family = "tiled";
            ok = ok || sh == FWI_SHAPE_TILED_ROWS8 || sh == FWI_SHAPE_TILED_ROWS4 ||
                 sh == FWI_SHAPE_TILED_QUADS;
        }
        if (!ok) {
            delete pl;
            return fail(FWI_ERR_UNSUPPORTED,
                        "shape %d is not a shape of the %s kernels this plan runs on", sh, family);
        }
    }
    if (fam == FWI_KERNELS_CLUSTER && !pl->cluster) {
        delete pl;
        return fail(FWI_ERR_UNSUPPORTED,
                    "the cluster kernels take 4th-order, whole-record plans of padded width <= %d "
                    "whose rows split over 2 to 8 CTAs' shared memory (grid %dx%d)",
                    fwi::kCluPitch - 4, pl->NZ, pl->NX);
    }
    // the adjoint source of a receiver enters through the level psi^{j-1}
    // scaled by 1/B, B = 1 - eta dt/2 of the receiver cell
    {
        const double lnR = std::log(1.0 / (double)p.refl_R);
        for (int i = 0; i < p.nr; ++i) {
            const int px = pl->rec_px[i], pz = pl->rec_pz[i];
            double cx = 0.0, cz = pz > p.nz - 1 ? pz - (p.nz - 1) : 0;
            if (px < p.nb) cx = p.nb - px;
            if (px > p.nb + p.nx - 1) cx = px - (p.nb + p.nx - 1);
            const double e = p.nb > 0 ? 3.0 * p.v_ref * lnR / p.nb *
                                            ((cx / p.nb) * (cx / p.nb) / p.dx +
                                             (cz / p.nb) * (cz / p.nb) / p.dz) * p.dt / 2.0
                                      : 0.0;
            if (std::fabs(1.0 - e) < 1e-3) {
                delete pl;
                return fail(FWI_ERR_UNSUPPORTED,
                            "receiver %d sits where the damping makes 1 - eta dt/2 vanish", i);
            }
        }
    }
    // the resident adjoint injects each receiver from the thread that owns
    // its cell: receivers must sit in distinct column strips
    for (int i = 0; i < ((pl->tiled || pl->cpml) ? 0 : p.nr); ++i)
        for (int k = 0; k < i; ++k)
            if (pl->rec_px[i] == pl->rec_px[k] &&
                pl->rec_pz[i] / pl->shape_adj.rows == pl->rec_pz[k] / pl->shape_adj.rows) {
                delete pl;
                return fail(FWI_ERR_UNSUPPORTED,
                            "receivers %d and %d share a column strip of %d rows", k, i,
                            pl->shape_adj.rows);
            }
    // W2 trace kernel shared memory
    if (fwi::w2_trace_smem(p.nt, w2->n_xi) > 227 * 1024) {
        delete pl;
        return fail(FWI_ERR_UNSUPPORTED, "nt + n_xi too large for the W2 trace kernel");
    }
    const size_t B = p.batch, ntr = (size_t)p.ns * p.nr;
    using fwi::align_up;
    size_t o = fwi::kStatusBytes;
    pl->ws_w2 = o;
    o += align_up(B * ntr * 4);
    pl->ws_gshot = o;
    o += align_up(B * p.ns * (size_t)p.nz * p.nx * 4);
    // record planes: nzs rows of pitch fast_PR (fast kernels), NX (generic)
    // or NXp (tiled)
    const size_t rec_plane = (size_t)pl->nzs * pl->rec_pitch * 4;
    const size_t cells = (size_t)pl->NZ * pl->NX;
    pl->ckpt_every = p.checkpoint_every > p.nt ? p.nt : p.checkpoint_every;
    pl->nslot = pl->ckpt_every ? (p.nt + pl->ckpt_every - 1) / pl->ckpt_every : 0;
    pl->ws_seg = pl->ws_astate = pl->ws_asrc = 0;
    if (pl->ckpt_every) {
        pl->ws_seg = o;       // one segment of the record
        o += align_up(B * p.ns * (size_t)pl->ckpt_every * rec_plane);
        if (!pl->tiled) {     // (the tiled adjoint keeps its state in its own fields)
            pl->ws_astate = o;    // adjoint levels j, j-1 and imaging sums
            o += align_up(B * p.ns * 3 * cells * 4);
            pl->ws_asrc = o;      // source-cell imaging sums
            o += align_up(B * p.ns * 4);
        }
    }
    pl->ws_t_u0 = pl->ws_t_u1 = pl->ws_t_v = pl->ws_t_p0 = pl->ws_t_p1 = pl->ws_t_w = 0;
    pl->ws_t_acc = 0;
    pl->ws_t_ka = pl->ws_t_ab = pl->ws_t_accsrc = pl->ws_t_rec = pl->ws_t_src = 0;
    if (pl->tiled) {
        const size_t field = align_up(B * p.ns * (size_t)pl->NZ * pl->NXp * 4);
        const size_t table = align_up(B * (size_t)pl->NZ * pl->NXp * 4);
        pl->ws_t_u0 = o;  o += field;
        pl->ws_t_u1 = o;  o += field;
        pl->ws_t_v = o;   o += field;
        pl->ws_t_p0 = o;  o += field;
        pl->ws_t_p1 = o;  o += field;
        pl->ws_t_w = o;   o += field;
        pl->ws_t_acc = o; o += field;
        pl->ws_t_ka = o;  o += table;
        pl->ws_t_ab = o;  o += table;
        pl->ws_t_accsrc = o; o += align_up(B * p.ns * 4);
        pl->ws_t_rec = o; o += align_up((size_t)p.nr * 4);
        pl->ws_t_src = o; o += align_up((size_t)p.ns * 4);
    }
    if (pl->cpml) {
        pl->ws_c = o;   // fields, memory variables, kappa and the layer profiles
        o += align_up(fwi::cpml_workspace(*pl));
    }
    pl->ws_bytes = o;
    o = 0;
    pl->ctx_M = o;      o += align_up(B * 4);
    pl->ctx_S = o;      o += align_up(B * 4);
    pl->ctx_S2 = o;     o += align_up(B * 4);
    pl->ctx_cshift = o; o += align_up(B * ntr * 4);
    pl->ctx_str = o;    o += align_up(B * ntr * 4);
    pl->ctx_omega = o;  o += align_up(B * ntr * p.nt * 4);
    pl->ctx_Qb = o;     o += align_up(B * ntr * w2->n_xi * 4);   // int bracket base
    pl->ctx_Qf = o;     o += align_up(B * ntr * w2->n_xi * 4);   // fraction in bracket
    pl->ctx_bytes = o;
    pl->snap_bytes = pl->ckpt_every ? (size_t)pl->nslot * B * p.ns * 2 * cells * 4
                                    : B * p.ns * (size_t)p.nt * rec_plane;
    *out = reinterpret_cast<fwi_plan *>(pl);
    return FWI_OK;
}

void fwi_plan_destroy(fwi_plan *plan) { delete reinterpret_cast<Plan *>(plan); }

fwi_status fwi_plan_sizes(const fwi_plan *plan, size_t *workspace_bytes, size_t *obs_ctx_bytes,
                          size_t *snapshot_bytes)
{
    if (!plan) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
    const Plan *pl = as_plan(plan);
    if (workspace_bytes) *workspace_bytes = pl->ws_bytes;
    if (obs_ctx_bytes) *obs_ctx_bytes = pl->ctx_bytes;
    if (snapshot_bytes) *snapshot_bytes = pl->snap_bytes;
    return FWI_OK;
}

fwi_status fwi_plan_padded(const fwi_plan *plan, int *NZ, int *NX)
{
    if (!plan) return fail(FWI_ERR_INVALID_ARG, "plan is NULL");
    if (NZ) *NZ = as_plan(plan)->NZ;
    if (NX) *NX = as_plan(plan)->NX;
    return FWI_OK;
}

fwi_status fwi_plan_kernels(const fwi_plan *plan, int *family)
{
    if (!plan || !family) return fail(FWI_ERR_INVALID_ARG, "plan or family is NULL");
    const Plan *pl = as_plan(plan);
    *family = pl->cpml      ? FWI_KERNELS_CPML
              : pl->cluster ? FWI_KERNELS_CLUSTER
              : pl->tiled   ? FWI_KERNELS_TILED
                            : FWI_KERNELS_RESIDENT;
    return FWI_OK;
}

fwi_status fwi_forward(const fwi_plan *plan, const float *v, float *d_syn, float *snapshots,
                       void *workspace, void *stream)
{
    if (!plan || !v || !d_syn || !workspace)
        return fail(FWI_ERR_INVALID_ARG, "plan, v, d_syn and workspace must not be NULL");
    if (misaligned16(snapshots) || misaligned16(workspace))
        return fail(FWI_ERR_INVALID_ARG, "snapshots and workspace must be 16-byte aligned");
    const Plan &pl = *as_plan(plan);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_forward status reset");
    if (pl.ckpt_every) {
        fwi::Window w;
        w.ckpt = snapshots;
        w.ckpt_every = pl.ckpt_every;
        e = fwi::launch_forward(pl, v, d_syn, nullptr, workspace, st, w);
    } else {
        e = fwi::launch_forward(pl, v, d_syn, snapshots, workspace, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fwi_forward launch");
    return FWI_OK;
}

fwi_status fwi_forward_wait_check(const fwi_plan *plan, const float *v, float *d_syn,
                                  float *snapshots, void *workspace, void *stream)
{
    if (!plan || !v || !d_syn || !workspace)
        return fail(FWI_ERR_INVALID_ARG, "plan, v, d_syn and workspace must not be NULL");
    if (misaligned16(snapshots) || misaligned16(workspace))
        return fail(FWI_ERR_INVALID_ARG, "snapshots and workspace must be 16-byte aligned");
    const Plan &pl = *as_plan(plan);
    if (!pl.cluster && !(pl.tiled && !pl.cpml))
        return fail(FWI_ERR_UNSUPPORTED,
                    "the wait self-check runs the cluster and tiled kernels only");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_forward_wait_check status reset");
    fwi::Window w;
    w.wait_check = true;
    e = fwi::launch_forward(pl, v, d_syn, snapshots, workspace, st, w);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_forward_wait_check launch");
    return FWI_OK;
}

fwi_status fwi_w2_prepare(const fwi_plan *plan, const float *d_obs, void *obs_ctx, void *stream)
{
    if (!plan || !d_obs || !obs_ctx)
        return fail(FWI_ERR_INVALID_ARG, "plan, d_obs and obs_ctx must not be NULL");
    cudaError_t e = fwi::launch_w2_prepare(*as_plan(plan), d_obs, (unsigned char *)obs_ctx,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_w2_prepare launch");
    return FWI_OK;
}

fwi_status fwi_w2_misfit(const fwi_plan *plan, const void *obs_ctx, const float *d_syn, float *J,
                         float *w2, float *adj_src, void *workspace, void *stream)
{
    if (!plan || !obs_ctx || !d_syn || !J || !workspace)
        return fail(FWI_ERR_INVALID_ARG,
                    "plan, obs_ctx, d_syn, J and workspace must not be NULL");
    const Plan &pl = *as_plan(plan);
    float *scratch = (float *)((unsigned char *)workspace + pl.ws_w2);
    cudaError_t e = fwi::launch_w2_misfit(pl, (const unsigned char *)obs_ctx, d_syn, J, w2,
                                          adj_src, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_w2_misfit launch");
    return FWI_OK;
}

fwi_status fwi_adjoint_grad(const fwi_plan *plan, const float *v, const float *adj_src,
                            const float *snapshots, float *grad, void *workspace, void *stream)
{
    if (!plan || !v || !adj_src || !snapshots || !grad || !workspace)
        return fail(FWI_ERR_INVALID_ARG,
                    "plan, v, adj_src, snapshots, grad and workspace must not be NULL");
    if (misaligned16(snapshots) || misaligned16(workspace))
        return fail(FWI_ERR_INVALID_ARG, "snapshots and workspace must be 16-byte aligned");
    const Plan &pl = *as_plan(plan);
    unsigned char *ws = (unsigned char *)workspace;
    float *gshot = (float *)(ws + pl.ws_gshot);
    cudaStream_t st = (cudaStream_t)stream;
    if (!pl.ckpt_every) {
        cudaError_t e = fwi::launch_adjoint(pl, v, adj_src, snapshots, grad, gshot, workspace, st);
        if (e != cudaSuccess) return cuda_fail(e, "fwi_adjoint_grad launch");
        return FWI_OK;
    }
    // checkpointed: segments of K forward steps, last first; each is
    // recomputed from its checkpoint into the segment record, then run
    // backwards with the adjoint state carried from the previous segment
    const int K = pl.ckpt_every, nt = pl.p.nt;
    const size_t slot = (size_t)pl.p.batch * pl.p.ns * 2 * pl.NZ * pl.NX;
    float *seg = (float *)(ws + pl.ws_seg);
    for (int sgi = pl.nslot - 1; sgi >= 0; --sgi) {
        const int fb = sgi * K, fe = fb + K < nt ? fb + K : nt;
        fwi::Window wf;
        wf.j_begin = fb;
        wf.j_end = fe;
        wf.rec_base = fb;
        wf.rec_planes = K;
        wf.resume = sgi > 0 ? snapshots + sgi * slot : nullptr;
        cudaError_t e = fwi::launch_forward(pl, v, nullptr, seg, workspace, st, wf);
        if (e != cudaSuccess) return cuda_fail(e, "fwi_adjoint_grad recompute launch");
        fwi::Window wa;
        wa.j_begin = nt - fe;
        wa.j_end = nt - fb;
        wa.rec_base = fb;
        wa.rec_planes = K;
        wa.astate = (float *)(ws + pl.ws_astate);
        wa.asrc = (float *)(ws + pl.ws_asrc);
        e = fwi::launch_adjoint(pl, v, adj_src, seg, grad, gshot, workspace, st, wa);
        if (e != cudaSuccess) return cuda_fail(e, "fwi_adjoint_grad launch");
    }
    return FWI_OK;
}

fwi_status fwi_guided_step(int batch, int nz, int nx, const fwi_guide_params *params,
                           const float *v_prime, const float *v0hat, const float *g,
                           const float *h, float *v_out, float *rho_out, void *stream)
{
    if (batch < 1 || nz < 1 || nx < 1) return fail(FWI_ERR_INVALID_ARG, "batch, nz, nx must be >= 1");
    if (!params || !v_prime || !v0hat || !g || !h || !v_out)
        return fail(FWI_ERR_INVALID_ARG, "params and array pointers must not be NULL");
    const fwi_guide_params &gp = *params;
    if (!(gp.c > 0.0) || !(gp.eps > 0.0) || !(gp.gamma >= 0.0) || !(gp.rho0 >= 0.0) ||
        !std::isfinite(gp.tau) || !finite_pos(gp.unit))
        return fail(FWI_ERR_INVALID_ARG,
                    "need c > 0, eps > 0, gamma >= 0, rho0 >= 0, finite tau, unit > 0");
    if ((size_t)nz * nx > (size_t)1 << 30) return fail(FWI_ERR_UNSUPPORTED, "grid too large");
    cudaError_t e = fwi::launch_guided(batch, nz, nx, gp, v_prime, v0hat, g, h, v_out, rho_out,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_guided_step launch");
    return FWI_OK;
}

fwi_status fwi_check(const fwi_plan *plan, void *workspace, void *stream)
{
    if (!plan || !workspace) return fail(FWI_ERR_INVALID_ARG, "plan and workspace must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, workspace, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_check");
    e = cudaMemsetAsync(workspace, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "fwi_check reset");
    if (code == FWI_ERR_UNSTABLE_CFL)
        return fail(FWI_ERR_UNSTABLE_CFL, "a velocity outside (0, v_max] reached the device");
    if (code == FWI_ERR_DEVICE_TIMEOUT)
        return fail(FWI_ERR_DEVICE_TIMEOUT, "a device-side wait ran out of its budget");
    if (code != 0) return fail((fwi_status)code, "device status %d", code);
    return FWI_OK;
}

}  // extern "C"
