"""Host-side checks of the build helpers: the kernel digest that ties a
committed profile to the code it measured ignores comments and whitespace
but not code, and the committed traffic record names a digest of that form."""
import json
import os

from paper_2211_12265_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_code_only_strips_comments_and_whitespace():
    a = "int x = 1; // one\n/* block\n comment */ int  y = 2;\n"
    b = "int x = 1;\nint y = 2;"
    assert build._code_only(a) == build._code_only(b) == "int x = 1; int y = 2;"
    assert build._code_only("int x = 1;") != build._code_only("int x = 2;")


def test_digest_is_stable_and_per_unit():
    d = build.source_digest()
    assert d == build.source_digest("dil_sign.cu") and len(d) == 16
    assert d != build.source_digest("dil_verify.cu")


def test_traffic_record_names_a_digest():
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_sign_level2_traffic.json")))
    assert len(rec["source_digest"]) == 16
    assert rec["dram_bytes_per_task"] == round((rec["dram_bytes_read"] + rec["dram_bytes_write"]) / rec["tasks_captured"])
