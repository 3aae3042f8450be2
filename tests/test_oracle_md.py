"""Pins for the oracle's velocity-Verlet integrator (the MD step around the
forces of Eq. 3): each test ties it to something other than itself -- the
CODATA constants as scipy holds them, free flight, one step of a dimer worked
out by hand from the closed-form dimer energy, time reversibility, energy and
momentum conservation, and the second-order error scaling of the method."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from scipy import constants

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

MASSES = np.array([72.63, 121.76, 127.60])


def tiny_hyper():
    return I.Hyper(n_types=3, n_rad=3, n_ang=2, k_rad=4, k_ang=3, l_max=4, has_4body=1, n_hidden=4,
                   rc_rad=5.0, rc_ang=4.0)


def small_packing(n=40, tag=81):
    return I.packing_batch([n], tag=tag)


def test_unit_factor_against_codata():
    """1 u A^2/fs^2 in eV = m_u * 1e-20 m^2 / 1e-30 s^2 / e: 103.6427 (the
    factor the MD workload states)."""
    want = constants.physical_constants["atomic mass constant"][0] * 1e10 / constants.e
    assert O.MVV_EV == pytest.approx(want, rel=1e-8)       # CODATA 2018 vs the release scipy holds
    assert O.MVV_EV == pytest.approx(103.6427, abs=5e-5)


def test_free_flight_and_wrap():
    """Atoms beyond each other's cutoff feel no force: x(t) = x0 + v t, and
    the wrap at the rebuild step maps them back into the box."""
    h = tiny_hyper()
    th = I.init_params(h, seed=3)
    L = 40.0
    pos = np.array([[1.0, 2.0, 3.0], [20.0, 21.0, 22.0], [39.5, 10.0, 0.2]])
    vel = np.array([[0.01, -0.02, 0.005], [-0.003, 0.0, 0.001], [0.05, 0.0, -0.02]])
    types = np.array([0, 1, 2])
    box, off = np.array([[L, L, L]]), np.array([0, 3])
    r = O.velocity_verlet(h, th, pos, vel, types, box, off, MASSES, 2.0, 12, rebuild_every=10)
    assert np.array_equal(r["vel"], vel)
    x = pos + 2.0 * 11 * vel                    # 11 drifts, then the wrap at step 10, then one more
    x = x - L * np.floor(x / L) + 2.0 * vel
    assert np.allclose(r["pos"], x, atol=1e-12)
    assert np.all(r["epot"] == r["epot"][0])


def _dimer_energy(h, prm, ta, tb, r):
    e = 0.0
    for a, b in ((ta, tb), (tb, ta)):
        qq = []
        for coef, rc in ((prm.cR[a, b], h.rc_rad), (prm.cA[a, b], h.rc_ang)):
            x = 2 * (r / rc - 1) ** 2 - 1
            fc = 0.5 * (1 + math.cos(math.pi * r / rc)) if r < rc else 0.0
            Q = np.array([0.5 * (npcheb.chebval(x, [0] * k + [1]) + 1) * fc for k in range(coef.shape[1])])
            qq.append(coef @ Q)
        gR, gA = qq
        q = np.concatenate([gR, np.repeat(gA ** 2, h.l_max), 2.0 / 9.0 * gA ** 3])
        e += prm.w1[a] @ np.tanh(prm.W0[a] @ q + prm.b0[a]) + prm.b1[a]
    return e


def test_one_dimer_step_by_hand():
    """One step of a Ge-Te dimer along z, with the force taken as the
    central difference of the closed-form dimer energy: half kick with
    a = F/(m 103.6427), drift, force at the new bond length, half kick."""
    h = tiny_hyper()
    th = I.init_params(h, seed=5)
    prm = O.unpack(h, th)
    ta, tb, r0, dt = 0, 2, 3.0, 2.0
    L = 50.0
    pos = np.array([[25.0, 25.0, 25.0], [25.0, 25.0, 25.0 + r0]])
    vel = np.array([[0.0, 0.0, 0.004], [0.0, 0.0, -0.001]])

    def fz(r):          # force on the second atom along +z
        return -(_dimer_energy(h, prm, ta, tb, r + 1e-6) - _dimer_energy(h, prm, ta, tb, r - 1e-6)) / 2e-6
    kappa = 103.6427
    m = MASSES[[ta, tb]]
    F0 = np.array([-fz(r0), fz(r0)])
    v = vel[:, 2] + 0.5 * dt * F0 / (m * kappa)
    z = pos[:, 2] + dt * v
    F1 = np.array([-fz(z[1] - z[0]), fz(z[1] - z[0])])
    v = v + 0.5 * dt * F1 / (m * kappa)
    r = O.velocity_verlet(h, th, pos, vel, np.array([ta, tb]), np.array([[L, L, L]]), np.array([0, 2]),
                          MASSES, dt, 1, rebuild_every=10)
    assert np.allclose(r["pos"][:, 2], z, rtol=0, atol=1e-9)
    assert np.allclose(r["vel"][:, 2], v, rtol=0, atol=1e-9)
    assert np.allclose(r["F"][:, 2], F1, rtol=0, atol=1e-7)
    assert np.all(r["pos"][:, :2] == 25.0) and np.all(r["vel"][:, :2] == 0.0)


def test_time_reversal():
    """Velocity Verlet is symmetric: n steps, velocities negated, n steps
    more return to the start (no wrap in between)."""
    h = tiny_hyper()
    th = I.init_params(h, seed=2)
    s = small_packing()
    v0 = I.maxwell_boltzmann(s.types, 900.0, atom_off=s.atom_off)
    x0 = s.pos.astype(np.float64)
    a = O.velocity_verlet(h, th, x0, v0, s.types, s.box, s.atom_off, MASSES, 2.0, 8, rebuild_every=1000)
    # the wrap at step 0 of the backward run moves nothing: re-wrap the forward end first
    xa = O.wrap_positions(a["pos"], s.box, s.atom_off)
    b = O.velocity_verlet(h, th, xa, -a["vel"], s.types, s.box, s.atom_off, MASSES, 2.0, 8,
                          rebuild_every=1000, force=a["F"])
    L = s.box[0]
    d = b["pos"] - x0
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9
    assert np.allclose(-b["vel"], v0, atol=1e-12)


def test_energy_momentum_conservation_and_second_order():
    """Total energy is conserved to O(dt^2) (halving dt cuts the fluctuation
    about four-fold) and the total momentum stays at zero (sum F = 0)."""
    h = tiny_hyper()
    th = I.init_params(h, seed=4)
    s = small_packing()
    v0 = I.maxwell_boltzmann(s.types, 900.0, atom_off=s.atom_off)
    dev = []
    for dt, n in ((2.0, 60), (1.0, 120)):
        r = O.velocity_verlet(h, th, s.pos, v0, s.types, s.box, s.atom_off, MASSES, dt, n)
        et = r["epot"][:, 0] + r["ekin"][:, 0]
        e0 = O.kinetic_energy(v0, s.types, MASSES, s.atom_off)[0] + \
            O.energy_forces_virial(h, th, s.pos, s.types, s.box, s.atom_off,
                                   O.neighbor_pairs(s.pos32(), s.box, s.atom_off, h.rc_rad))["Etot"][0]
        dev.append(np.abs(et - e0).max() / s.n_atoms)
        p = (MASSES[s.types][:, None] * r["vel"]).sum(0)
        assert np.abs(p).max() < 1e-12
    assert dev[0] < 1e-4
    assert 2.5 < dev[0] / dev[1] < 6.0
