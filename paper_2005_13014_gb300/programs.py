"""The stencil programs of this library in the textual stencil-program form.

The form restates the paper's stencil dialect (§IV): ``input`` fields are
loaded (stencil.load), each ``stage`` is one stencil.apply whose body reads
earlier values at constant offsets (stencil.access) and returns its results
(stencil.return), ``column ... = thomas(a, b, c, d...)`` solves a tridiagonal
system along k in every (i, j) column, and ``output`` values are stored over
the domain (stencil.store). ``kpos`` is the level index relative to the
domain's lower k bound and ``ksize`` the domain's extent in k.

``oec_program_create`` recognises these three programs (by structure, not by
text) and runs them with the hand-written kernels; other programs go through
the generic code generator.
"""

# Horizontal diffusion (the shape Table II lists as hdiffsa): 5-point Laplacian,
# i/j fluxes with a sign limiter, flux divergence.
HDIFF = """
input in, coeff
stage lap = 4.0*in - in[-1,0,0] - in[1,0,0] - in[0,-1,0] - in[0,1,0]
stage flx = { let f = lap[1,0,0] - lap; return select(f*(in[1,0,0] - in) > 0.0, 0.0, f) }
stage fly = { let f = lap[0,1,0] - lap; return select(f*(in[0,1,0] - in) > 0.0, 0.0, f) }
stage out = in - coeff*((flx - flx[-1,0,0]) + (fly - fly[0,-1,0]))
output out
"""


def _hdiff_of(x, tag):
    return f"""
stage lap{tag} = 4.0*{x} - {x}[-1,0,0] - {x}[1,0,0] - {x}[0,-1,0] - {x}[0,1,0]
stage flx{tag} = {{ let f = lap{tag}[1,0,0] - lap{tag}; return select(f*({x}[1,0,0] - {x}) > 0.0, 0.0, f) }}
stage fly{tag} = {{ let f = lap{tag}[0,1,0] - lap{tag}; return select(f*({x}[0,1,0] - {x}) > 0.0, 0.0, f) }}
stage {x}d = {x} - coeff*((flx{tag} - flx{tag}[-1,0,0]) + (fly{tag} - fly{tag}[0,-1,0]))
"""


# Horizontal diffusion of u and v followed by implicit vertical advection: one
# tridiagonal system per (i, j) column (staggered wind wf = (w + w(i+1))/2),
# solved by the Thomas algorithm (§VII-B) for both right-hand sides.
HDIFF_VADVC = ("""
input u, v, w, coeff
param dtr
""" + _hdiff_of("u", "u") + _hdiff_of("v", "v") + """
stage wf = 0.5*(w + w[1,0,0])
stage a = select(kpos > 0.0, -0.25*wf, 0.0)
stage c = select(kpos < ksize - 1.0, 0.25*wf[0,0,1], 0.0)
stage b = dtr + abs(a) + abs(c)
stage du = dtr*ud - 0.5*(select(kpos > 0.0, a*(ud[0,0,-1] - ud), 0.0) + select(kpos < ksize - 1.0, c*(ud[0,0,1] - ud), 0.0))
stage dv = dtr*vd - 0.5*(select(kpos > 0.0, a*(vd[0,0,-1] - vd), 0.0) + select(kpos < ksize - 1.0, c*(vd[0,0,1] - vd), 0.0))
column u_out, v_out = thomas(a, b, c, du, dv)
output u_out, v_out
""")

# Fastwaves-like program (the shape Table II lists as fastwavesuv: six applies,
# nine inputs, two outputs, no control flow): vertical pressure interpolation,
# its k difference, terrain-following pressure gradients in i and j, a
# fourth-order divergence, and the wind update.
FASTWAVES = """
input u_in, v_in, utens, vtens, pp, rho, wgtfac, hhl, fx
param dt, alpha
stage ppgk = wgtfac*pp + (1.0 - wgtfac)*pp[0,0,-1]
stage ppgc = ppgk[0,0,1] - ppgk
stage ppgu = (pp[1,0,0] - pp) + 0.25*(ppgc[1,0,0] + ppgc)*((hhl[0,0,1] + hhl) - (hhl[1,0,1] + hhl[1,0,0])) / ((hhl[0,0,1] - hhl) + (hhl[1,0,1] - hhl[1,0,0]))
stage ppgv = (pp[0,1,0] - pp) + 0.25*(ppgc[0,1,0] + ppgc)*((hhl[0,0,1] + hhl) - (hhl[0,1,1] + hhl[0,1,0])) / ((hhl[0,0,1] - hhl) + (hhl[0,1,1] - hhl[0,1,0]))
stage div = (-u_in[2,0,0] + 8.0*u_in[1,0,0] - 8.0*u_in[-1,0,0] + u_in[-2,0,0])/12.0 + (-v_in[0,2,0] + 8.0*v_in[0,1,0] - 8.0*v_in[0,-1,0] + v_in[0,-2,0])/12.0
stage u_out, v_out = { return u_in + dt*((utens - ppgu*2.0*fx/(rho[1,0,0] + rho)) + alpha*(div[1,0,0] - div)), v_in + dt*((vtens - ppgv*2.0*fx/(rho[0,1,0] + rho)) + alpha*(div[0,1,0] - div)) }
output u_out, v_out
"""

BUILTIN = {"hdiff": HDIFF, "hdiff_vadvc": HDIFF_VADVC, "fastwaves": FASTWAVES}

# ---- shape-matched stand-ins for more of the paper's test set (Table II) ----
# The paper gives only the shape of its COSMO/FV3 benchmarks (applies,
# inputs/outputs, control flow), not their formulas; these programs have the
# listed shapes with stencils of the same kind (averaging, pressure gradients
# over a k-staggered grid, third- and fifth-order upwind advection with an
# `if` written as select, a clipped Smagorinsky coefficient, interface values
# and upwind flux selection), and run through the generic code generator.
# Every select decides on an input field, never on a computed value, so FP32
# and FP64 take the same branch. They are stand-ins, not the COSMO/FV3
# kernels. With hdiff (hdiffsa) and fastwaves (fastwavesuv) they cover all
# eleven rows of Table II.

# uvbke (FV3): 2 applies, 4 inputs / 2 outputs
UVBKE = """
input uc, vc, cosa, rsina
param dt5
stage ub = dt5*(uc[0,-1,0] + uc - (vc[-1,0,0] + vc)*cosa)*rsina
stage vb = dt5*(vc[-1,0,0] + vc - (uc[0,-1,0] + uc)*cosa)*rsina
output ub, vb
"""

# p_grad_c (FV3): 3 applies, 7 inputs / 2 outputs, 3-D (k-staggered pressure)
P_GRAD_C = """
input uc, vc, delpc, pkc, gz, rdxc, rdyc
param dt2
stage wk = delpc + pkc[0,0,1] - pkc
stage uc_out = uc + dt2*rdxc/(wk[-1,0,0] + wk)*((gz[-1,0,1] - gz)*(pkc[0,0,1] - pkc[-1,0,0]) + (gz[-1,0,0] - gz[0,0,1])*(pkc[-1,0,1] - pkc))
stage vc_out = vc + dt2*rdyc/(wk[0,-1,0] + wk)*((gz[0,-1,1] - gz)*(pkc[0,0,1] - pkc[0,-1,0]) + (gz[0,-1,0] - gz[0,0,1])*(pkc[0,-1,1] - pkc))
output uc_out, vc_out
"""

# hadvuv (COSMO): 8 applies, 6 inputs / 2 outputs, `if` (upwind direction)
HADVUV = """
input uin, vin, uatupos, vatupos, uatvpos, vatvpos
param eddlat, eddlon
stage axu = if (uatupos > 0.0) { yield uatupos*(2.0*uin[1,0,0] + 3.0*uin - 6.0*uin[-1,0,0] + uin[-2,0,0]) } else { yield uatupos*(-uin[2,0,0] + 6.0*uin[1,0,0] - 3.0*uin - 2.0*uin[-1,0,0]) }
stage ayu = if (vatupos > 0.0) { yield vatupos*(2.0*uin[0,1,0] + 3.0*uin - 6.0*uin[0,-1,0] + uin[0,-2,0]) } else { yield vatupos*(-uin[0,2,0] + 6.0*uin[0,1,0] - 3.0*uin - 2.0*uin[0,-1,0]) }
stage axv = if (uatvpos > 0.0) { yield uatvpos*(2.0*vin[1,0,0] + 3.0*vin - 6.0*vin[-1,0,0] + vin[-2,0,0]) } else { yield uatvpos*(-vin[2,0,0] + 6.0*vin[1,0,0] - 3.0*vin - 2.0*vin[-1,0,0]) }
stage ayv = if (vatvpos > 0.0) { yield vatvpos*(2.0*vin[0,1,0] + 3.0*vin - 6.0*vin[0,-1,0] + vin[0,-2,0]) } else { yield vatvpos*(-vin[0,2,0] + 6.0*vin[0,1,0] - 3.0*vin - 2.0*vin[0,-1,0]) }
stage advu = (eddlon*axu + eddlat*ayu)/6.0
stage advv = (eddlon*axv + eddlat*ayv)/6.0
stage uout = uin - advu
stage vout = vin - advv
output uout, vout
"""

# fvtp2d_flux (FV3): 5 applies, 7 inputs / 2 outputs, `if` (upwind side)
FVTP2D_FLUX = """
input q, crx, cry, xfx, yfx, al, bl
stage qm = 0.5*(q[1,0,0] + q[-1,0,0])
stage fx1 = if (crx > 0.0) { yield q[-1,0,0] + (1.0 - crx)*(al - q[-1,0,0]) } else { yield q + (1.0 + crx)*(al - qm) }
stage fy1 = if (cry > 0.0) { yield q[0,-1,0] + (1.0 - cry)*(bl - q[0,-1,0]) } else { yield q + (1.0 + cry)*(bl - q) }
stage fx = xfx*fx1
stage fy = yfx*fy1
output fx, fy
"""

# hdiffsmag (COSMO): 6 applies, 8 inputs / 2 outputs, min/max (Smagorinsky
# coefficient clipped to [0, 0.5]; the deformation enters squared)
HDIFFSMAG = """
input u, v, hdmask, crlavo, crlavu, crlato, crlatu, acrlat0
param eddlat, eddlon, tau_smag, weight_smag
stage t = eddlon*(u - u[-1,0,0]) - eddlat*acrlat0*(v - v[0,-1,0])
stage s = eddlat*crlavo*(u[0,1,0] - u) + eddlon*(v[1,0,0] - v)
stage smag_u = min(0.5, max(0.0, tau_smag*(t*t + s[0,-1,0]*s[0,-1,0]) - weight_smag))
stage smag_v = min(0.5, max(0.0, tau_smag*(t[0,1,0]*t[0,1,0] + s[-1,0,0]*s[-1,0,0]) - weight_smag))
stage u_out = u + hdmask*smag_u*(u[1,0,0] + u[-1,0,0] - 2.0*u + crlato*(u[0,1,0] - u) + crlatu*(u[0,-1,0] - u))
stage v_out = v + hdmask*smag_v*(v[1,0,0] + v[-1,0,0] - 2.0*v + crlavo*(v[0,1,0] - v) + crlavu*(v[0,-1,0] - v))
output u_out, v_out
"""

# hadvuv5th (COSMO): 8 applies, 6 inputs / 2 outputs, `if` (upwind
# direction), fifth-order upwind stencils (offsets up to 3)
HADVUV5TH = """
input uin, vin, uatupos, vatupos, uatvpos, vatvpos
param eddlat, eddlon
stage axu = if (uatupos > 0.0) { yield uatupos*(-2.0*uin[-3,0,0] + 15.0*uin[-2,0,0] - 60.0*uin[-1,0,0] + 20.0*uin + 30.0*uin[1,0,0] - 3.0*uin[2,0,0]) } else { yield uatupos*(3.0*uin[-2,0,0] - 30.0*uin[-1,0,0] - 20.0*uin + 60.0*uin[1,0,0] - 15.0*uin[2,0,0] + 2.0*uin[3,0,0]) }
stage ayu = if (vatupos > 0.0) { yield vatupos*(-2.0*uin[0,-3,0] + 15.0*uin[0,-2,0] - 60.0*uin[0,-1,0] + 20.0*uin + 30.0*uin[0,1,0] - 3.0*uin[0,2,0]) } else { yield vatupos*(3.0*uin[0,-2,0] - 30.0*uin[0,-1,0] - 20.0*uin + 60.0*uin[0,1,0] - 15.0*uin[0,2,0] + 2.0*uin[0,3,0]) }
stage axv = if (uatvpos > 0.0) { yield uatvpos*(-2.0*vin[-3,0,0] + 15.0*vin[-2,0,0] - 60.0*vin[-1,0,0] + 20.0*vin + 30.0*vin[1,0,0] - 3.0*vin[2,0,0]) } else { yield uatvpos*(3.0*vin[-2,0,0] - 30.0*vin[-1,0,0] - 20.0*vin + 60.0*vin[1,0,0] - 15.0*vin[2,0,0] + 2.0*vin[3,0,0]) }
stage ayv = if (vatvpos > 0.0) { yield vatvpos*(-2.0*vin[0,-3,0] + 15.0*vin[0,-2,0] - 60.0*vin[0,-1,0] + 20.0*vin + 30.0*vin[0,1,0] - 3.0*vin[0,2,0]) } else { yield vatvpos*(3.0*vin[0,-2,0] - 30.0*vin[0,-1,0] - 20.0*vin + 60.0*vin[0,1,0] - 15.0*vin[0,2,0] + 2.0*vin[0,3,0]) }
stage advu = (eddlon*axu + eddlat*ayu)/60.0
stage advv = (eddlon*axv + eddlat*ayv)/60.0
stage uout = uin - advu
stage vout = vin - advv
output uout, vout
"""

# nh_p_grad (FV3): 5 applies, 8 inputs / 2 outputs, 3-D (non-hydrostatic
# pressure gradient over a k-staggered grid)
NH_P_GRAD = """
input u, v, rdx, rdy, gz, pp, pk3, delp
param dt
stage wk = pk3[0,0,1] - pk3
stage du = dt/(wk + wk[1,0,0])*((gz[0,0,1] - gz[1,0,0])*(pk3[1,0,1] - pk3) + (gz - gz[1,0,1])*(pk3[0,0,1] - pk3[1,0,0]))
stage dv = dt/(wk + wk[0,1,0])*((gz[0,0,1] - gz[0,1,0])*(pk3[0,1,1] - pk3) + (gz - gz[0,1,1])*(pk3[0,0,1] - pk3[0,1,0]))
stage u_out = (u + du*rdx) + dt*rdx*(pp[1,0,0] - pp)/(delp + delp[1,0,0])
stage v_out = (v + dv*rdy) + dt*rdy*(pp[0,1,0] - pp)/(delp + delp[0,1,0])
output u_out, v_out
"""

# fvtp2d_qi (FV3): 5 applies, 5 inputs / 2 outputs, `if` (upwind side):
# fourth-order interface values along i, an upwind flux, the flux-form update
FVTP2D_QI = """
input q, crx, xfx, area, ra_x
stage al = 0.5833333333333334*(q[-1,0,0] + q) - 0.08333333333333333*(q[-2,0,0] + q[1,0,0])
stage bl = al - q
stage br = al[1,0,0] - q
stage fx1 = if (crx > 0.0) { yield q[-1,0,0] + (1.0 - crx)*(br[-1,0,0] - crx*(bl[-1,0,0] + br[-1,0,0])) } else { yield q + (1.0 + crx)*(bl + crx*(bl + br)) }
stage q_i = (q*area + fx1*xfx - fx1[1,0,0]*xfx[1,0,0])/ra_x
output fx1, q_i
"""

# fvtp2d_qj (FV3): 8 applies, 6 inputs / 3 outputs, `if` (upwind side):
# as fvtp2d_qi along j, with a smoothness bound and a mass flux
FVTP2D_QJ = """
input q, cry, yfx, area, ra_y, mfy
stage al = 0.5833333333333334*(q[0,-1,0] + q) - 0.08333333333333333*(q[0,-2,0] + q[0,1,0])
stage bl = al - q
stage br = al[0,1,0] - q
stage b0 = min(abs(bl), abs(br))*(bl + br)
stage fy1 = if (cry > 0.0) { yield q[0,-1,0] + (1.0 - cry)*(br[0,-1,0] - cry*b0[0,-1,0]) } else { yield q + (1.0 + cry)*(bl + cry*b0) }
stage fy = yfx*fy1
stage q_j = (q*area + fy - fy[0,1,0])/ra_y
stage mf = mfy*fy1
output fy, q_j, mf
"""

# name: (text, scalar parameters, (applies, inputs, outputs) as Table II lists them)
TESTSET = {
    "uvbke": (UVBKE, [0.5], (2, 4, 2)),
    "p_grad_c": (P_GRAD_C, [0.01], (3, 7, 2)),
    "hadvuv": (HADVUV, [0.1, 0.1], (8, 6, 2)),
    "fvtp2d_flux": (FVTP2D_FLUX, [], (5, 7, 2)),
    "hdiffsmag": (HDIFFSMAG, [0.5, 0.5, 0.1, 0.01], (6, 8, 2)),
    "hadvuv5th": (HADVUV5TH, [0.1, 0.1], (8, 6, 2)),
    "nh_p_grad": (NH_P_GRAD, [0.01], (5, 8, 2)),
    "fvtp2d_qi": (FVTP2D_QI, [], (5, 5, 2)),
    "fvtp2d_qj": (FVTP2D_QJ, [], (8, 6, 3)),
}

# default scalar parameters of the synthetic workloads
PARAMS = {"hdiff": [], "hdiff_vadvc": [2.0], "fastwaves": [0.5, 0.0625]}
