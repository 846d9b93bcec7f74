// builtin_programs.h - the textual form of the programs that have hand-written
// kernels. oec_program_create compares the canonical form of a parsed program
// with these to pick the hand-written kernel family.
#pragma once

namespace oec {

static const char* const kBuiltin_hdiff = R"OEC(
input in, coeff
stage lap = 4.0*in - in[-1,0,0] - in[1,0,0] - in[0,-1,0] - in[0,1,0]
stage flx = { let f = lap[1,0,0] - lap; return select(f*(in[1,0,0] - in) > 0.0, 0.0, f) }
stage fly = { let f = lap[0,1,0] - lap; return select(f*(in[0,1,0] - in) > 0.0, 0.0, f) }
stage out = in - coeff*((flx - flx[-1,0,0]) + (fly - fly[0,-1,0]))
output out
)OEC";

static const char* const kBuiltin_hdiff_vadvc = R"OEC(
input u, v, w, coeff
param dtr

stage lapu = 4.0*u - u[-1,0,0] - u[1,0,0] - u[0,-1,0] - u[0,1,0]
stage flxu = { let f = lapu[1,0,0] - lapu; return select(f*(u[1,0,0] - u) > 0.0, 0.0, f) }
stage flyu = { let f = lapu[0,1,0] - lapu; return select(f*(u[0,1,0] - u) > 0.0, 0.0, f) }
stage ud = u - coeff*((flxu - flxu[-1,0,0]) + (flyu - flyu[0,-1,0]))

stage lapv = 4.0*v - v[-1,0,0] - v[1,0,0] - v[0,-1,0] - v[0,1,0]
stage flxv = { let f = lapv[1,0,0] - lapv; return select(f*(v[1,0,0] - v) > 0.0, 0.0, f) }
stage flyv = { let f = lapv[0,1,0] - lapv; return select(f*(v[0,1,0] - v) > 0.0, 0.0, f) }
stage vd = v - coeff*((flxv - flxv[-1,0,0]) + (flyv - flyv[0,-1,0]))

stage wf = 0.5*(w + w[1,0,0])
stage a = select(kpos > 0.0, -0.25*wf, 0.0)
stage c = select(kpos < ksize - 1.0, 0.25*wf[0,0,1], 0.0)
stage b = dtr + abs(a) + abs(c)
stage du = dtr*ud - 0.5*(select(kpos > 0.0, a*(ud[0,0,-1] - ud), 0.0) + select(kpos < ksize - 1.0, c*(ud[0,0,1] - ud), 0.0))
stage dv = dtr*vd - 0.5*(select(kpos > 0.0, a*(vd[0,0,-1] - vd), 0.0) + select(kpos < ksize - 1.0, c*(vd[0,0,1] - vd), 0.0))
column u_out, v_out = thomas(a, b, c, du, dv)
output u_out, v_out
)OEC";

static const char* const kBuiltin_fastwaves = R"OEC(
input u_in, v_in, utens, vtens, pp, rho, wgtfac, hhl, fx
param dt, alpha
stage ppgk = wgtfac*pp + (1.0 - wgtfac)*pp[0,0,-1]
stage ppgc = ppgk[0,0,1] - ppgk
stage ppgu = (pp[1,0,0] - pp) + 0.25*(ppgc[1,0,0] + ppgc)*((hhl[0,0,1] + hhl) - (hhl[1,0,1] + hhl[1,0,0])) / ((hhl[0,0,1] - hhl) + (hhl[1,0,1] - hhl[1,0,0]))
stage ppgv = (pp[0,1,0] - pp) + 0.25*(ppgc[0,1,0] + ppgc)*((hhl[0,0,1] + hhl) - (hhl[0,1,1] + hhl[0,1,0])) / ((hhl[0,0,1] - hhl) + (hhl[0,1,1] - hhl[0,1,0]))
stage div = (-u_in[2,0,0] + 8.0*u_in[1,0,0] - 8.0*u_in[-1,0,0] + u_in[-2,0,0])/12.0 + (-v_in[0,2,0] + 8.0*v_in[0,1,0] - 8.0*v_in[0,-1,0] + v_in[0,-2,0])/12.0
stage u_out, v_out = { return u_in + dt*((utens - ppgu*2.0*fx/(rho[1,0,0] + rho)) + alpha*(div[1,0,0] - div)), v_in + dt*((vtens - ppgv*2.0*fx/(rho[0,1,0] + rho)) + alpha*(div[0,1,0] - div)) }
output u_out, v_out
)OEC";

}  // namespace oec
