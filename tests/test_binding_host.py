"""Host-side checks of the Python binding (no GPU): every array it hands to the library
as a raw device pointer is checked first, since the library reads a fixed number of
values from it and cannot check the buffer itself."""
import numpy as np
import pytest

from paper_2604_19723_gb300 import bp

torch = pytest.importorskip("torch")

J, NZ = 4, 160
FLOATS = 2 * J * NZ


def problem(**kw):
    args = dict(is_tensor=True, is_cuda=True, on_current_device=True, contiguous=True, dtype="complex64",
                shape=(J, NZ), want_dtypes=("complex64", "float32"), want_floats=FLOATS, want_cols=None)
    args.update(kw)
    return bp.device_array_problem(**args)


def test_accepts_the_observation_forms_the_callers_use():
    assert problem() is None                                            # J x Nz complex64
    assert problem(dtype="float32", shape=(J, NZ, 2)) is None           # J x Nz x 2 float32
    assert problem(dtype="float32", shape=(FLOATS,)) is None            # a batch row of z_floats()
    assert problem(dtype="float32", shape=(200, 16), want_dtypes=("float32",), want_floats=3200,
                   want_cols=16) is None                                # network inputs


@pytest.mark.parametrize("kw, words", [
    (dict(is_tensor=False), "torch tensor"),
    (dict(is_cuda=False), "CUDA"),
    (dict(on_current_device=False), "another device"),
    (dict(dtype="complex128"), "dtype"),
    (dict(dtype="float64", shape=(J, NZ, 2)), "dtype"),
    (dict(contiguous=False), "contiguous"),
    (dict(shape=(J - 1, NZ)), "values"),                  # too short: the library would read past it
    (dict(shape=(J + 1, NZ)), "values"),                  # too long: a shape mistake
    (dict(dtype="float32", shape=(J, NZ)), "values"),     # complex data passed as its real parts
    (dict(dtype="float32", shape=(200, 8), want_dtypes=("float32",), want_floats=1600, want_cols=16), "shape"),
])
def test_rejects_what_the_library_cannot_read_safely(kw, words):
    p = problem(**kw)
    assert p is not None and words in p, p


def test_host_tensors_and_other_objects_raise_invalid_argument():
    for bad in (torch.zeros((J, NZ), dtype=torch.complex64), np.zeros((J, NZ), np.complex64), None):
        with pytest.raises(bp.BPError) as e:
            bp._device_array(bad, "bp_update: z", ("complex64", "float32"), FLOATS)
        assert e.value.status == 1 and "bp_update: z" in str(e.value)
