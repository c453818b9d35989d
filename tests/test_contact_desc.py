"""Host-side marshalling of contacts and attachments into the C ABI's
pd_contact_desc (no GPU: the descriptor is read back through its own
pointers), and the attachment targets' schedule (Sec. 4.6)."""
import ctypes

import numpy as np
import pytest

from paper_2605_14526_b300 import binding, inputs


def _spec():
    return inputs.ContactSpec(ground=np.array([3, 1, 4]), box=np.array([9]), ground_z=-0.5, box_z0=0.3,
                              box_travel=0.02, box_steps=5, mu=0.4, attach=np.array([7, 2]),
                              attach_p0=np.array([[0.1, 0.2, 0.3], [1.0, 2.0, 3.0]]),
                              attach_travel=np.array([[0.0, 0.0, 0.01], [0.02, 0.0, 0.0]]), attach_steps=4)


def _read(ptr, ctype, n):
    return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), shape=(n,)).copy()


def test_descriptor_points_at_the_spec_arrays():
    spec = _spec()
    desc, keep = binding.contact_desc(spec, tol=1e-10, max_iters=77)
    assert (desc.n_ground, desc.n_box, desc.n_attach) == (3, 1, 2)
    assert np.array_equal(_read(desc.ground, ctypes.c_int32, 3), [3, 1, 4])
    assert np.array_equal(_read(desc.box, ctypes.c_int32, 1), [9])
    assert np.array_equal(_read(desc.attach, ctypes.c_int32, 2), [7, 2])
    assert np.array_equal(_read(desc.attach_target, ctypes.c_double, 6), spec.attach_p0.ravel())
    assert np.array_equal(_read(desc.attach_travel, ctypes.c_double, 6), spec.attach_travel.ravel())
    assert (desc.ground_z, desc.box_z0, desc.box_travel, desc.box_steps) == (-0.5, 0.3, 0.02, 5)
    assert (desc.mu, desc.tol, desc.max_iters, desc.attach_steps) == (0.4, 1e-10, 77, 4)


def test_descriptor_without_attachments_has_null_arrays():
    spec = _spec()
    spec.attach, spec.attach_p0, spec.attach_travel = np.zeros(0, dtype=np.int64), np.zeros((0, 3)), np.zeros((0, 3))
    desc, keep = binding.contact_desc(spec)
    assert desc.n_attach == 0 and not desc.attach and not desc.attach_target and not desc.attach_travel


def test_descriptor_rejects_mismatched_target_rows():
    spec = _spec()
    spec.attach_p0 = spec.attach_p0[:1]
    with pytest.raises(ValueError):
        binding.contact_desc(spec)


def test_attachment_targets_move_linearly_then_hold():
    spec = _spec()
    p0, tr = spec.attach_p0, spec.attach_travel
    for t in range(8):
        assert np.allclose(spec.attach_target(t), p0 + min(t + 1, 4) / 4 * tr, rtol=0, atol=1e-15)
    spec.attach_steps = 0    # refused, as pd_set_contacts refuses it
    with pytest.raises(ValueError):
        spec.attach_target(0)
