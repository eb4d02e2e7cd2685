"""The log-Cholesky inertia randomisation of the input generator (CPU): exact round trip
at zero noise, and every sample physically consistent (positive mass, positive-definite
pseudo-inertia, inertia about the centre of mass positive definite and obeying the
triangle inequalities)."""
import numpy as np

from paper_2601_22074_b300 import inputs as I


def test_round_trip_and_consistency():
    for spec in (I.quadruped(), I.humanoid()):
        x0 = I.randomised_inertia(spec, 2, 0, 0.0)
        np.testing.assert_allclose(x0[0, :, 0], spec.body_mass, atol=1e-12)
        np.testing.assert_allclose(x0[0, :, 1:4], spec.body_ipos, atol=1e-12)
        np.testing.assert_allclose(x0[0, :, 4:], spec.body_inertia, atol=1e-12)
        x = I.randomised_inertia(spec, 64, 1, 0.3)
        for w in range(64):
            for b in range(1, spec.nbody):
                m, c, I6 = x[w, b, 0], x[w, b, 1:4], x[w, b, 4:]
                assert m > 0
                J = I.inertia_to_pseudo(m, c, I6)
                assert np.linalg.eigvalsh(J).min() > 0
                Ic = np.array([[I6[0], I6[3], I6[4]], [I6[3], I6[1], I6[5]], [I6[4], I6[5], I6[2]]])
                ev = np.linalg.eigvalsh(Ic)
                assert ev.min() > 0
                assert ev[0] + ev[1] >= ev[2] * (1 - 1e-9)
