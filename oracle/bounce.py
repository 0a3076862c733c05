"""Bounce-back rules for a wall at an arbitrary fraction of a lattice link
(oracle, FP64, numpy; test infrastructure only).

A boundary node B lies q Delta from a flat wall along a link that crosses it
(q = d_w for every crossing link of a wall parallel to the lattice planes).
For a direction i pointing into the wall, opp(i) is the population entering
the fluid at B; F = B - c_i is the next fluid node along the link.

Inputs per crossing direction (post-collision values of the previous step):
  fs_i_B   f*_i(x_B, t)
  fs_i_F   f*_i(x_F, t)       (equal to f_i(x_B, t+1) after streaming)
  fs_o_B   f*_opp(i)(x_B, t)  (equal to f_opp(i)(x_F, t+1) after streaming)
  mw       2 w_i rho_w c_i . u_w / c_s^2, the moving-wall term of Eq. 31.
Each rule returns f_opp(i)(x_B, t+1).
"""
from __future__ import annotations


def halfway(fs_i_B, mw):
    """Eq. 31 (q = 1/2)."""
    return fs_i_B - mw


def bouzidi(q, fs_i_B, fs_i_F, fs_o_B, mw):
    """Eq. 36 (Bouzidi et al.).  q >= 1/2: the reflected population is
    interpolated between the bounced-back f*_i(B) and f_opp(F, t+1); q < 1/2:
    the population reaching the wall is interpolated between f*_i(B) and
    f*_i(F) before it is bounced back.  Both branches give Eq. 31 at q = 1/2."""
    if q >= 0.5:
        return fs_i_B / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fs_o_B - mw / (2.0 * q)
    return 2.0 * q * fs_i_B + (1.0 - 2.0 * q) * fs_i_F - mw


def yu(q, fs_i_B, fs_i_F, fs_o_B, mw):
    """Eq. 37 (Yu et al.), one expression for every q.

    First line (reading): the population of direction i that reaches the wall
    point W at t+1, linearly interpolated along the link between its value
    streamed into B, f_i(x_B, t+1) = f*_i(x_F, t), and the value f*_i(x_B, t)
    that streams on past B (weights 1 - q and q), is bounced back with the
    moving-wall term.  The printed line is garbled; this is Yu et al.'s
    construction, and it keeps f_opp(x_F, t+1) in the result at q = 1/2 as the
    text says.  Second line as printed: B lies between W (distance q) and F
    (distance 1), so the value at B is interpolated with weight q / (1 + q)."""
    f_W = (1.0 - q) * fs_i_F + q * fs_i_B - mw
    return f_W + (q / (q + 1.0)) * (fs_o_B - f_W)


RULES = {"bouzidi": bouzidi, "yu": yu}
