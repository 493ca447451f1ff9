"""The public device header (include/gga_device.cuh) is enough on its own to
build a user's kernels: the user library compiles for sm_103a with only
include/ on the include path, and needs nothing from the GGArray library
(no GPU needed here)."""

import re
import subprocess

from user_kernel import build_user


def test_user_kernels_build_against_the_public_header_alone():
    path = build_user()
    defined = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in ["user_push_rounds", "user_push_rounds_cursor", "user_push_own", "user_push_formula", "user_read_global", "user_read_local", "user_push_rejected"]:
        assert re.search(r"\bT\s+" + name + r"\b", defined), name
    undefined = subprocess.run(["nm", "-D", "--undefined-only", path], capture_output=True, text=True).stdout
    assert "gga_" not in undefined
