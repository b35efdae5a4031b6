// res_finish.cuh -- the df64 outer residual's totals from its block partials (device code shared by
// k_mixed.cu, which finishes right after the residual, and k_poisson.cu, whose refinement-loop
// condition kernel finishes them in the captured step).  Include after df64.cuh and
// envar_internal.cuh.
#pragma once

namespace envar {

// The residual's totals of member m from its n block partials, by one warp (lane l takes partials
// l, l + 32, ...; the maximum is exact in any order, the df64 sum is lane 0's butterfly total):
// max |r| with the convergence test against rtol_abs (outer_done, inner_done, the refinement
// count), and the fluid sum of x.  Members already converged are left alone.
__device__ __forceinline__ void res_finish_member(const RedCtx &rc, MemberCtl *ctl, int m, int n, double rtol_abs, int count_it)
{
    const int lane = threadIdx.x & 31;
    if (ctl[m].outer_done) return;
    const double *pm = rc.part + ((long long)RS_RMAX * rc.stride + m) * rc.nblk;
    const double *ps = rc.part + ((long long)RS_XSUM * rc.stride + m) * rc.nblk;
    float mx = 0.f;
    f2 xs{0.f, 0.f};
    for (int q = lane; q < n; q += 32) {
        mx = fmaxf(mx, __ldcg(reinterpret_cast<const float *>(pm + q)));
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(ps + q));
        xs = df_add(xs, f2{v.x, v.y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    xs = warp_sum_df(xs);
    if (lane == 0) {
        const double tot = (double)mx;
        rc.red[m].val[RS_RMAX] = tot;
        rc.red[m].val[RS_XSUM] = df_to_d(xs);
        const int done = (tot <= rtol_abs) ? 1 : 0;
        ctl[m].outer_done = done;
        ctl[m].inner_done = done;
        if (!done && count_it) ctl[m].outer_its += 1;
    }
}

} // namespace envar
