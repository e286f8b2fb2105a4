"""The oracle's pins catch plausible mistakes: each case plants one mistake in the oracle's source
(a dropped term or factor, a wrong sign or index, a transposed or unconjugated operand) and runs
the pin files against it in a child process, which must end with a failed assertion.  The stored
goldens are left out of these runs, since they were written by the oracle itself; what catches a
mistake here is the mathematics the pins check (closed forms, the direct DFT, dense
diagonalisation, Courant-Fischer bounds, invariances, brute force).

Mistakes that change only how fast an iteration converges, not what it converges to (the sign
of the PCG conjugacy ratio, the choice of half set, the dropping threshold), and rewrites that
compute the same thing (a wider enumeration margin around the sphere, another valid round-robin
order), are not listed: the pins fix results, not speed or form.
"""
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["tests/test_oracle_hamiltonian.py", "tests/test_oracle_solvers.py", "tests/test_oracle_next.py"]
SELF_REFERENTIAL = ["tests/test_oracle_solvers.py::test_golden_files_reproduce"]

# (name, module, text in the oracle, planted replacement)
MUTANTS = [
    # plane-wave sphere and kinetic energy (Sec. 2.1)
    ("kinetic_drops_half", "oracle.basis", "return 0.5 * np.einsum", "return np.einsum"),
    ("kinetic_wrong_k_sign", "oracle.basis", "dtype=np.float64) + np.asarray(kpt", "dtype=np.float64) - np.asarray(kpt"),
    ("sphere_wrong_k_sign", "oracle.basis", "d = n + k[None, :]", "d = n - k[None, :]"),
    ("sphere_drops_points_on_the_edge", "oracle.basis", "<= r2 + 1e-9", "< r2 - 1e-9"),
    ("sphere_radius_without_2pi", "oracle.basis", "(a / (2.0 * math.pi)) ** 2", "(a / math.pi) ** 2"),
    ("box_index_negated", "oracle.basis", "np.mod(np.asarray(miller), N)", "np.mod(-np.asarray(miller), N)"),
    # local potential and Kleinman-Bylander terms (Sec. 2.2 items iii, iv)
    ("dft_wrong_exponent_sign", "oracle.hamiltonian", "np.exp(-2j * np.pi * np.outer(j, j) / N)",
     "np.exp(2j * np.pi * np.outer(j, j) / N)"),
    ("dft_wrong_normalisation", "oracle.hamiltonian", "return t / N ** 3", "return t / N ** 2"),
    ("dense_H_transposed_index", "oracle.hamiltonian", "n[:, None, :] - n[None, :, :]", "n[None, :, :] - n[:, None, :]"),
    ("dense_H_drops_kinetic", "oracle.hamiltonian", "H = H + np.diag(basis.kinetic(n, kpt, a))", "H = H + 0.0"),
    ("dense_H_unconjugated_projector", "oracle.hamiltonian", "@ beta.conj().T", "@ beta.T"),
    ("dense_H_drops_kb_energies", "oracle.hamiltonian", "(beta * E[None, :]) @", "beta @"),
    ("fft_route_wrong_sign", "oracle.hamiltonian", "psi = scipy.fft.ifftn(box, axes=(0, 1, 2), norm=\"forward\"",
     "psi = scipy.fft.fftn(box, axes=(0, 1, 2), norm=\"backward\""),
    ("fft_route_wrong_normalisation", "oracle.hamiltonian", "Vpsi = scipy.fft.fftn(psi, axes=(0, 1, 2), norm=\"forward\"",
     "Vpsi = scipy.fft.fftn(psi, axes=(0, 1, 2), norm=\"backward\""),
    ("fft_route_unconjugated_projector", "oracle.hamiltonian", "B = self.beta.conj().T @ X", "B = self.beta.T @ X"),
    ("apply_drops_kinetic", "oracle.hamiltonian", "Y = self.T[:, None] * X + self.apply_local(X)", "Y = self.apply_local(X)"),
    ("apply_wrong_kb_sign", "oracle.hamiltonian", "+ self.apply_nonlocal(X)", "- self.apply_nonlocal(X)"),
    ("kpoint_always_the_first", "oracle.hamiltonian", "kpt = w.kpts[k_index]", "kpt = w.kpts[0]"),
    ("projectors_of_the_first_kpoint", "oracle.hamiltonian", "beta = w.beta(miller, k_index) if w.nproj",
     "beta = w.beta(miller, 0) if w.nproj"),
    # the Lanczos route
    ("lanczos_largest_instead_of_smallest", "oracle.lanczos", 'which="SA"', 'which="LA"'),
    ("lanczos_descending_order", "oracle.lanczos", "order = np.argsort(w)", "order = np.argsort(-w)"),
    # Jacobi rotations
    ("jacobi_wrong_rotation_sign", "oracle.jacobi", "u_qp, u_qq = -s * np.conj(ph)", "u_qp, u_qq = s * np.conj(ph)"),
    ("jacobi_conjugated_phase", "oracle.jacobi", "ph = np.where(act, b / np.where", "ph = np.where(act, np.conj(b) / np.where"),
    ("jacobi_stop_test_inverted", "oracle.jacobi", "if off <= tol * scale:", "if off >= tol * scale:"),
    # block LOBPCG (Algorithm 1, Sec. 3.2) and the Teter ratio
    ("teter_wrong_power", "oracle.lobpcg", "p / (p + 16.0 * x ** 4)", "p / (p + 16.0 * x ** 3)"),
    ("teter_wrong_coefficient", "oracle.lobpcg", "12.0 + 8.0 * x", "12.0 + 6.0 * x"),
    ("ekin_not_normalised", "oracle.lobpcg", "/ np.einsum(\"gi->i\", np.abs(X) ** 2)", ""),
    ("constraint_unconjugated", "oracle.lobpcg", "V = V - Y @ (Y.conj().T @ V)", "V = V - Y @ (Y.T @ V)"),
    ("gram_unconjugated", "oracle.lobpcg", "A = Z.conj().T @ HZ", "A = Z.T @ HZ"),
    ("gram_symmetrised_without_conjugate", "oracle.lobpcg", "S = 0.5 * (S + S.conj().T)", "S = 0.5 * (S + S.T)"),
    ("ritz_vectors_miss_the_scaling", "oracle.lobpcg", "C = d[:, None] * (B @ Q[:, :m])", "C = B @ Q[:, :m]"),
    ("rr_basis_not_orthonormalised", "oracle.lobpcg", "B = U[:, keep] / np.sqrt(mu[keep])[None, :]", "B = U[:, keep]"),
    ("block_not_constrained", "oracle.lobpcg", "X = orthonormalize(project_out(Y, X))", "X = orthonormalize(X)"),
    ("direction_not_constrained", "oracle.lobpcg", "W = project_out(Y, W)", "W = W"),
    ("coefficients_swapped", "oracle.lobpcg", "Cx, Cw = C[:m], C[m:2 * m]", "Cx, Cw = C[m:2 * m], C[:m]"),
    ("residual_wrong_sign", "oracle.lobpcg", "R = HX - X * theta[None, :]", "R = HX + X * theta[None, :]"),
    ("search_direction_drops_p", "oracle.lobpcg", "Pn, HPn = Pn + P @ Cp, HPn + HP @ Cp", "Pn, HPn = Pn, HPn"),
    ("p_is_the_previous_w", "oracle.lobpcg", "P, HP = Pn, HPn", "P, HP = W, HW"),
    ("final_rr_not_applied_to_hx", "oracle.lobpcg", "X, HX = X @ C, HX @ C\n        nrm", "X, HX = X @ C, HX\n        nrm"),
    ("ritz_pairs_from_the_top", "oracle.lobpcg", "return theta[:m], C", "return theta[-m:], d[:, None] * (B @ Q[:, -m:])"),
    ("constraint_misses_the_previous_block", "oracle.lobpcg", "Y = X[:, :b * block] if b else None",
     "Y = X[:, :(b - 1) * block] if b > 1 else None"),
    ("converged_on_the_smallest_residual", "oracle.lobpcg", "if rc.max() <= tol:", "if rc.min() <= tol:"),
    ("convergence_looks_at_the_buffer_bands", "oracle.lobpcg", "rc = r if nconv is None else r[:nconv]",
     "rc = r if nconv is None else r[nconv:]"),
    # density (Sec. 2.1)
    ("density_direct_wrong_sign", "oracle.density", "np.exp(2j * np.pi * (j @ n.T) / N)", "np.exp(-2j * np.pi * (j @ n.T) / N)"),
    ("density_direct_wrong_volume", "oracle.density", "reshape(N, N, N) / a ** 3", "reshape(N, N, N) / a ** 2"),
    ("density_drops_occupation", "oracle.density", "rho += float(f[b]) * (", "rho += ("),
    ("density_wrong_modulus", "oracle.density", "psi.real ** 2 + psi.imag ** 2", "psi.real ** 2 - psi.imag ** 2"),
    ("electron_count_wrong_cell", "oracle.density", "* a ** 3 / N ** 3", "* a ** 3 / N ** 2"),
    ("density_fft_route_wrong_volume", "oracle.density", "return rho / a ** 3", "return rho / a ** 2"),
    ("density_fft_route_conjugated_band", "oracle.density", "box[idx] = C[:, b]", "box[idx] = np.conj(C[:, b])"),
    # Gamma-point real form
    ("half_set_misses_the_z_axis", "oracle.gamma", "if x > 0 or (x == 0 and (y > 0 or (y == 0 and z > 0))):",
     "if x > 0 or (x == 0 and y > 0):"),
    ("real_basis_wrong_sign", "oracle.gamma", "U[minus, 1 + h + cols] = -1j * s", "U[minus, 1 + h + cols] = 1j * s"),
    ("real_basis_wrong_norm", "oracle.gamma", "s = 1.0 / np.sqrt(2.0)", "s = 0.5"),
    ("from_half_unconjugated", "oracle.gamma", "c[minus] = np.conj(h[1:])", "c[minus] = h[1:]"),
    ("half_inner_drops_the_pair_factor", "oracle.gamma", "2.0 * np.real(ha[1:]", "np.real(ha[1:]"),
    ("half_inner_drops_g0", "oracle.gamma", "return np.outer(ha[0].real, hb[0].real) + 2.0",
     "return 0.0 * np.outer(ha[0].real, hb[0].real) + 2.0"),
    ("real_H_unconjugated", "oracle.gamma", "y = self.U.conj().T @ self.H.apply", "y = self.U.T @ self.H.apply"),
    ("to_half_takes_the_other_half", "oracle.gamma", "c[zero:zero + 1], c[plus]]", "c[zero:zero + 1], c[minus]]"),
    ("real_kinetic_unconjugated", "oracle.gamma", "np.einsum(\"gi,g,gi->i\", self.U.conj(), H.T, self.U)",
     "np.einsum(\"gi,g,gi->i\", self.U, H.T, self.U)"),
    # band-by-band PCG (Sec. 3.3)
    ("line_angle_not_halved", "oracle.pcg", "theta = 0.5 * np.arctan2(-2.0 * C, B - A)", "theta = np.arctan2(-2.0 * C, B - A)"),
    ("pcg_band_not_normalised", "oracle.pcg", "x = x / np.linalg.norm(x)\n    hx = H.apply(x)", "hx = H.apply(x)"),
    ("line_minimum_finds_the_maximum", "oracle.pcg", "np.arctan2(-2.0 * C, B - A)", "np.arctan2(2.0 * C, B - A)"),
    ("line_energy_drops_the_factor", "oracle.pcg", "2.0 * C * s * c", "C * s * c"),
    ("line_uses_the_wrong_diagonal", "oracle.pcg", "B = float(np.real(np.vdot(dh, hd)))", "B = float(np.real(np.vdot(dh, dh)))"),
    ("line_wrong_coupling_sign", "oracle.pcg", "C = float(np.real(np.vdot(x, hd)))", "C = -float(np.real(np.vdot(x, hd)))"),
    ("pcg_direction_not_constrained", "oracle.pcg", "eta = project_out(Y, eta)", "eta = eta"),
    ("pcg_step_wrong_sign", "oracle.pcg", "x, hx = c * x + s * dh, c * hx + s * hd", "x, hx = c * x - s * dh, c * hx - s * hd"),
    ("pcg_constraint_misses_the_previous_band", "oracle.pcg", "X[:, :n] if n else None", "X[:, :n - 1] if n > 1 else None"),
    # comparisons
    ("projector_distance_unconjugated", "oracle.checks", "A - B @ (B.conj().T @ A)", "A - B @ (B.T @ A)"),
    ("residuals_not_normalised", "oracle.checks", "X = X / np.linalg.norm(X, axis=0)[None, :]", "X = X"),
    ("miller_map_unsorted", "oracle.checks", "return order[pos]", "return pos"),
    ("orthonormality_smallest_deviation", "oracle.checks", "np.eye(X.shape[1])).max())", "np.eye(X.shape[1])).min())"),
    ("orthonormality_unconjugated", "oracle.checks", "np.abs(X.conj().T @ X - np.eye", "np.abs(X.T @ X - np.eye"),
    ("clusters_split_inside_the_gap", "oracle.checks", "eig[i] - eig[i - 1] > gap", "eig[i] - eig[i - 1] >= 10 * gap"),
]


def _pytest_cmd():
    cmd = [sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-rfE", "-p", "tests._oracle_mutant", "-m", "not gpu"]
    for t in SELF_REFERENTIAL:
        cmd += ["--deselect", t]
    return cmd


def _run(mutant):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    env.pop("ORACLE_MUTANT", None)
    if mutant is not None:
        env["ORACLE_MUTANT"] = json.dumps(list(mutant[1:]))
    p = subprocess.run(_pytest_cmd(), cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def runs():
    cases = [None] + MUTANTS
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        out = list(ex.map(_run, cases))
    return {("clean" if c is None else c[0]): r for c, r in zip(cases, out)}


def test_every_planted_text_occurs_once():
    for name, mod, old, new in MUTANTS:
        path = os.path.join(ROOT, *mod.split(".")) + ".py"
        with open(path) as f:
            assert f.read().count(old) == 1, name
        assert old != new, name


def test_pins_pass_on_the_oracle_as_it_is(runs):
    rc, out = runs["clean"]
    assert rc == 0, out[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_the_planted_mistake(runs, name):
    rc, out = runs[name]
    # exit code 1: a test failed (2 and above would be a collection or usage error)
    assert rc == 1, out[-3000:]
    failed = [ln for ln in out.splitlines() if ln.startswith("FAILED")]
    assert failed, out[-3000:]
