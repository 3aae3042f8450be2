"""The pins bind: each test plants one plausible mistake in the oracle (on
the CPU, by replacing one of its functions for the duration of the test)
and checks that a pin in tests/test_oracle_pins.py or tests/test_train_loop.py
then fails."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import nep_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location("_mut_" + name, os.path.join(HERE, name + ".py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


P = _load("test_oracle_pins")
TL = _load("test_train_loop")


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_cutoff_with_the_wrong_sign_is_caught(monkeypatch):
    """f_c = (1 - cos(pi r/rc))/2 instead of (1 + cos)/2 (Eq. 14)."""
    def wrong(r, rc):
        inside = r < rc
        fc = np.where(inside, 0.5 * (1.0 - np.cos(np.pi * r / rc)), 0.0)
        dfc = np.where(inside, 0.5 * np.pi / rc * np.sin(np.pi * r / rc), 0.0)
        return fc, dfc
    monkeypatch.setattr(O, "cutoff_fn", wrong)
    _fails(P.test_cutoff_values)
    _fails(P.test_dimer_closed_form, 0, 2)


def test_chebyshev_index_shift_is_caught(monkeypatch):
    """Q_k built from T_{k+1} instead of T_k (Eq. 12)."""
    real = O.chebyshev_basis

    def wrong(r, rc, K):
        Q, dQ = real(r, rc, K + 1)
        return Q[..., 1:], dQ[..., 1:]
    monkeypatch.setattr(O, "chebyshev_basis", wrong)
    _fails(P.test_chebyshev_basis_against_library_and_cosines)
    _fails(P.test_dimer_closed_form, 1, 1)


def test_legendre_recursion_error_is_caught(monkeypatch):
    """Bonnet's recursion with (2l+1) in place of (2l-1)."""
    def wrong(c, L):
        Pl = [np.ones_like(c), c]
        dP = [np.zeros_like(c), np.ones_like(c)]
        for l in range(2, L + 1):
            Pl.append(((2 * l + 1) * c * Pl[l - 1] - (l - 1) * Pl[l - 2]) / l)
            dP.append(dP[l - 2] + (2 * l - 1) * Pl[l - 1])
        return Pl, dP
    monkeypatch.setattr(O, "legendre", wrong)
    _fails(P.test_legendre_against_scipy)
    _fails(P.test_legendre_form_equals_sform_addition_theorem)


def test_swapped_species_pair_is_caught(monkeypatch):
    """c indexed by (Zj, Zi) instead of (Zi, Zj)."""
    real = O._type_pair_apply
    monkeypatch.setattr(O, "_type_pair_apply", lambda coef, ti, tj, X: real(coef, tj, ti, X))
    _fails(P.test_dimer_closed_form, 0, 2)


def test_force_sign_flip_is_caught(monkeypatch):
    """F_i = +dE/dr_i instead of -dE/dr_i (Eq. 3)."""
    real = O.energy_forces_virial

    def wrong(*a, **k):
        out = dict(real(*a, **k))
        out["F"] = -out["F"]
        return out
    monkeypatch.setattr(O, "energy_forces_virial", wrong)
    _fails(P.test_forces_central_difference, "tiny")


def test_transposed_virial_sign_is_caught(monkeypatch):
    """V = +sum f (x) r instead of -sum f (x) r (Eq. 4)."""
    real = O.energy_forces_virial

    def wrong(*a, **k):
        out = dict(real(*a, **k))
        out["V"] = -out["V"]
        return out
    monkeypatch.setattr(O, "energy_forces_virial", wrong)
    _fails(P.test_virial_finite_strain)


def test_dropped_images_are_caught(monkeypatch):
    """Pairs through periodic images dropped (only the zero image kept)."""
    real = O.neighbor_pairs

    def wrong(*a, **k):
        i, j, s = real(*a, **k)
        keep = np.all(s == 0, axis=1)
        return i[keep], j[keep], s[keep]
    monkeypatch.setattr(O, "neighbor_pairs", wrong)
    _fails(P.test_neighbors_small_box_counts_images)


def test_loss_without_the_batch_mean_is_caught(monkeypatch):
    """The batch sum in place of the batch mean (Eqs. 18-21)."""
    real = O.loss_value

    def wrong(h, theta, pos, types, box, atom_off, *rest, **k):
        return real(h, theta, pos, types, box, atom_off, *rest, **k) * (len(atom_off) - 1)
    monkeypatch.setattr(O, "loss_value", wrong)
    _fails(P.test_loss_closed_form)


def test_adam_without_bias_correction_is_caught(monkeypatch):
    """Adam's first and second moments used without the 1 - beta^t corrections."""
    def wrong(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        return theta - lr * m / (np.sqrt(v) + eps), m, v
    monkeypatch.setattr(O, "adam_step", wrong)
    _fails(TL.test_oracle_adam_first_step_and_constant_gradient)


def test_pair_vector_sign_flip_is_caught(monkeypatch):
    """r_ij = r_i - r_j (images likewise) in place of r_j - r_i (Eq. 3)."""
    real = O.pair_vectors
    monkeypatch.setattr(O, "pair_vectors", lambda pos, box, i, j, s: -real(pos, box, i, j, s))
    _fails(P.test_forces_central_difference, "tiny")


def test_image_shift_with_the_wrong_sign_is_caught(monkeypatch):
    """r_ij = r_j - s L - r_i: the periodic image taken on the wrong side."""
    monkeypatch.setattr(O, "pair_vectors", lambda pos, box, i, j, s: (pos[j] - pos[i]) - s * box[i])
    _fails(P.test_rotation_translation_permutation_invariance)


def test_basis_derivative_without_the_chain_factor_is_caught(monkeypatch):
    """dQ_k/dr with dT_k/dx not multiplied by dx/dr (Eqs. 12-13)."""
    def wrong(r, rc, K):
        r = np.asarray(r, np.float64)
        fc, dfc = O.cutoff_fn(r, rc)
        x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
        T = np.polynomial.chebyshev.chebvander(x, K - 1)
        dT = np.stack([np.polynomial.chebyshev.chebval(x, np.polynomial.chebyshev.chebder(np.eye(K)[k]))
                       for k in range(K)], -1)
        return 0.5 * (T + 1.0) * fc[..., None], 0.5 * dT * fc[..., None] + 0.5 * (T + 1.0) * dfc[..., None]
    monkeypatch.setattr(O, "chebyshev_basis", wrong)
    _fails(P.test_forces_central_difference, "tiny")


def test_legendre_derivative_error_is_caught(monkeypatch):
    """P'_l = P'_{l-2} + (2l+1) P_{l-1}: the values right, the derivatives wrong."""
    def wrong(c, L):
        Pl = [np.ones_like(c), c]
        dP = [np.zeros_like(c), np.ones_like(c)]
        for l in range(2, L + 1):
            Pl.append(((2 * l - 1) * c * Pl[l - 1] - (l - 1) * Pl[l - 2]) / l)
            dP.append(dP[l - 2] + (2 * l + 1) * Pl[l - 1])
        return Pl, dP
    monkeypatch.setattr(O, "legendre", wrong)
    _fails(P.test_legendre_against_scipy)
    _fails(P.test_forces_central_difference, "tiny")


def test_adam_with_eps_inside_the_root_is_caught(monkeypatch):
    """lr mhat / sqrt(vhat + eps) in place of lr mhat / (sqrt(vhat) + eps)."""
    def wrong(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh, vh = m / (1 - beta1 ** t), v / (1 - beta2 ** t)
        return theta - lr * mh / np.sqrt(vh + eps), m, v
    monkeypatch.setattr(O, "adam_step", wrong)
    _fails(TL.test_oracle_adam_first_step_and_constant_gradient)


def test_loss_mode1_with_the_mode0_energy_term_is_caught(monkeypatch):
    """Mode 1's energy term (dE_b)^2/N_b replaced by mode 0's (dE_b/N_b)^2 (Eq. 19)."""
    real = O.loss_value

    def wrong(*a, mode=0, **k):
        return real(*a, mode=0 if mode == 1 else mode, **k)
    monkeypatch.setattr(O, "loss_value", wrong)
    _fails(P.test_loss_closed_form)


def test_empty_configuration_left_out_of_the_mean_is_caught(monkeypatch):
    """An empty configuration dropped from B as well as from the sum."""
    real = O.loss_value

    def wrong(h, theta, pos, types, box, atom_off, *rest, **k):
        n_cfg = len(atom_off) - 1
        n_full = int(np.count_nonzero(np.diff(atom_off)))
        return real(h, theta, pos, types, box, atom_off, *rest, **k) * n_cfg / max(n_full, 1)
    monkeypatch.setattr(O, "loss_value", wrong)
    _fails(P.test_loss_with_an_empty_configuration)


def test_swapped_network_bias_blocks_are_caught(monkeypatch):
    """unpack reading w1 where b0 sits and b0 where w1 sits."""
    real = O.unpack

    def wrong(h, theta):
        p = real(h, theta)
        return O.Params(p.W0, p.w1, p.b0, p.b1, p.cR, p.cA)
    monkeypatch.setattr(O, "unpack", wrong)
    _fails(P.test_unpack_follows_the_header_block_order)


def test_transposed_w0_block_is_caught(monkeypatch):
    """unpack reading each W0[t] as [D][H] and transposing it."""
    real = O.unpack

    def wrong(h, theta):
        p = real(h, theta)
        T, H, D = p.W0.shape
        return O.Params(p.W0.reshape(T, D, H).transpose(0, 2, 1).copy(), p.b0, p.w1, p.b1, p.cR, p.cA)
    monkeypatch.setattr(O, "unpack", wrong)
    _fails(P.test_unpack_follows_the_header_block_order)


def test_swapped_c_blocks_are_caught(monkeypatch):
    """unpack taking cR's species pair as (Zj, Zi)."""
    real = O.unpack

    def wrong(h, theta):
        p = real(h, theta)
        return O.Params(p.W0, p.b0, p.w1, p.b1, p.cR.transpose(1, 0, 2, 3).copy(), p.cA)
    monkeypatch.setattr(O, "unpack", wrong)
    _fails(P.test_unpack_follows_the_header_block_order)


MD = _load("test_oracle_md")


def test_wrong_unit_factor_is_caught(monkeypatch):
    """a = F m 103.6427 / 1e4 instead of F / (m 103.6427)."""
    monkeypatch.setattr(O, "MVV_EV", 1e4 / 103.6427)
    _fails(MD.test_unit_factor_against_codata)
    _fails(MD.test_one_dimer_step_by_hand)


def test_wrong_mass_index_is_caught(monkeypatch):
    """Each species integrated with the next species' mass."""
    real = O.velocity_verlet

    def wrong(h, theta, pos, vel, types, box, atom_off, masses, *a, **k):
        return real(h, theta, pos, vel, types, box, atom_off, np.roll(np.asarray(masses), 1), *a, **k)
    monkeypatch.setattr(O, "velocity_verlet", wrong)
    _fails(MD.test_one_dimer_step_by_hand)


def test_full_kick_before_drift_is_caught(monkeypatch):
    """Symplectic Euler (a full kick, then the drift) in place of velocity
    Verlet's two half kicks."""
    def wrong(h, theta, pos, vel, types, box, atom_off, masses, dt, n_steps, rebuild_every=10, force=None):
        pos, vel = np.array(pos, np.float64), np.array(vel, np.float64)
        inv_m = 1.0 / (np.asarray(masses, np.float64)[types] * O.MVV_EV)

        def forces(x):
            pr = O.neighbor_pairs(x.astype(np.float32), box, atom_off, h.rc_rad)
            out = O.energy_forces_virial(h, theta, x, types, box, atom_off, pr)
            return out["F"], out["Etot"]
        F = np.array(force, np.float64) if force is not None else forces(pos)[0]
        epot, ekin = [], []
        for k in range(n_steps):
            vel = vel + dt * F * inv_m[:, None]
            pos = pos + dt * vel
            if k % rebuild_every == 0:
                pos = O.wrap_positions(pos, box, atom_off)
            F, E = forces(pos)
            epot.append(E)
            ekin.append(O.kinetic_energy(vel, types, masses, atom_off))
        return dict(pos=pos, vel=vel, F=F, epot=np.array(epot), ekin=np.array(ekin))
    monkeypatch.setattr(O, "velocity_verlet", wrong)
    _fails(MD.test_one_dimer_step_by_hand)
    _fails(MD.test_time_reversal)
