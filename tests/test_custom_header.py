"""The user-defined walk header compiles for sm_103a (CPU only: nvcc
cross-compiles the test walk types without a GPU)."""
import custom_build


def test_custom_walks_compile(tmp_path):
    obj = custom_build.build(str(tmp_path), link=False)
    assert obj.endswith(".o")
