"""Helpers shared by the GPU tests: oracle runs that mirror a Grid's setup."""
import numpy as np

import oracle as O
from paper_2501_06377_gb300.sft import FlowParams


def oracle_params(fp: FlowParams) -> O.Params:
    return O.Params(d0=fp.d0, d2=fp.d2, d4=fp.d4, m1=fp.m1, m3=fp.m3, m5=fp.m5, nu=fp.nu,
                    adv_space=fp.adv_space, adv_time=fp.adv_time,
                    diffusion=fp.diffusion if fp.diffusion in ("rkl2", "rkg2") else "off",
                    advection=fp.advection, alpha_uw=fp.alpha_uw, safety=fp.cfl_safety,
                    eps_w="h" if fp.eps_w <= 0 else fp.eps_w, atten_b0=fp.atten_b0,
                    splitting=fp.splitting, nu_grid_alpha=fp.nu_grid_alpha)


def oracle_run(shape, fp, B0, t_target, max_steps=None):
    g = O.Grid(*shape)
    r = O.Realization(g, oracle_params(fp), np.asarray(B0, dtype=np.float64))
    r.advance(t_target, max_steps)
    return r


def params_from_draw(draw, **kw):
    d0, d2, d4, m1, m3, m5, nu = draw
    return FlowParams(d0=d0, d2=d2, d4=d4, m1=m1, m3=m3, m5=m5, nu=nu, **kw)


def rel_linf(a, b):
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / np.abs(b).max())
