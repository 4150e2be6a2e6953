"""The C ABI library loads without a GPU and exports every entry point that
include/hf.h declares, with the signatures the binding uses."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_05017_b300 import _binding, build
    build.build()
    return _binding.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hf_density_build", "hf_part_create", "hf_fieldset_build", "hf_fieldset_compute",
                     "hf_query", "hf_query_batch", "hf_torque", "hf_resample", "hf_rfft3d", "hf_fields"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1711_05017_b300 import _binding
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _binding.SIGNATURES, f"binding lacks {name}"


def test_version_and_error_string_without_gpu(lib):
    assert lib.hf_version().decode().startswith("hf ")
    assert isinstance(lib.hf_last_error(), bytes)


def test_scratch_sizes_are_host_only(lib):
    for n in (32, 64, 96, 128):
        he = n * n * (n // 2 + 1)
        assert lib.hf_rfft3d_scratch_bytes(n) >= 2 * he * 8
        assert lib.hf_fields_scratch_bytes(n) >= 3 * he * 8 + 3 * n**3 * 4
    assert lib.hf_rfft3d_scratch_bytes(100) == 0
